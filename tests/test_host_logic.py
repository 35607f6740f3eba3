"""Host-side logic of the benchmark and the workload generators (no GPU).

- Algorithmic bytes per node update: every stored population read once and
  written once (3Q values of 4 or 8 bytes; the 16-bit formats keep 3(Q-1)
  moving populations in 2 bytes and the three rest populations in 4).
- The traffic lookup scales the captured DRAM bytes per node to the bench
  lattice and refuses captures of another kernel source or another
  configuration.
- The contact-angle sweep is seeded (identical on every call), has the stated
  size range and total, and every member gets an admissible target pair.
"""
import json
import os

import numpy as np
import pytest

import bench
from paper_1511_02155_gb300 import workloads as W


def test_bytes_per_node():
    assert bench.bytes_per_node(19, "fp32") == 2 * 3 * 19 * 4 == 456
    assert bench.bytes_per_node(19, "fp64") == 912
    assert bench.bytes_per_node(19, "fp16") == bench.bytes_per_node(19, "bf16") == 2 * (3 * 18 * 2 + 3 * 4) == 240
    assert bench.bytes_per_node(9, "fp32") == 216
    assert bench.bytes_per_node(9, "fp16") == 120


def test_traffic_lookup_scales_and_refuses_stale_captures(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.json").write_text(json.dumps({
        "fused:spinodal256:fp32:0,0": {"source_sha256": "abc", "dram_bytes_per_node": 470.5},
    }))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_from_profiles("fused:spinodal256:fp32:0,0", "abc", 1000) == 470500
    assert bench.traffic_from_profiles("fused:spinodal256:fp32:0,0", "other", 1000) is None
    assert bench.traffic_from_profiles("fused:probe8192:fp32:0,0", "abc", 1000) is None


def test_committed_traffic_entries_are_well_formed():
    with open(os.path.join(os.path.dirname(__file__), "..", "profiles", "traffic.json")) as f:
        d = json.load(f)
    for tag, e in d.items():
        if tag.startswith("_"):
            continue
        assert e["dram_bytes_per_node"] == pytest.approx((e["dram_read_bytes"] + e["dram_write_bytes"]) / e["nodes"])
        assert len(e["source_sha256"]) == 64


def test_sweep_is_seeded_and_within_its_ranges():
    a = W.sweep_wells(96)
    b = W.sweep_wells(96)
    assert len(a) == 96
    nodes = 0
    for ma, mb in zip(a, b):
        assert ma["nx"] == mb["nx"] and np.array_equal(ma["solid"], mb["solid"])
        assert ma["angles"] == mb["angles"]
        assert 128 <= ma["nx"] <= 768 and ma["nx"] % 32 == 0 and ma["ny"] == ma["nx"] // 2
        assert all(30 <= t < 150 for pair in ma["angles"] for t in pair)
        C = np.stack(ma["C"])
        fluid = ma["solid"] == 0
        assert np.allclose(C.sum(0)[fluid], 1.0)  # concentrations sum to one in the fluid
        nodes += ma["nx"] * ma["ny"]
    assert 10e6 < nodes < 12.5e6


def test_every_sweep_member_has_an_admissible_target():
    tl = pytest.importorskip("paper_1511_02155_gb300")
    try:
        tl.load_library(build_if_missing=True)
    except Exception as e:  # pragma: no cover - no toolkit
        pytest.skip(f"libtlbm.so unavailable: {e}")
    for m in W.sweep_wells(96):
        ok = False
        for pair in m["angles"]:
            try:
                h = tl.wetting_from_angles(m["kappa"], m["alpha"], *pair)
            except tl.TLBMError:
                continue
            assert all(abs(4 * hm) < m["alpha"] * km for hm, km in zip(h, m["kappa"]))
            ok = True
            break
        assert ok


@pytest.mark.parametrize("theta", [20.0, 45.0, 80.0, 90.0, 100.0, 135.0, 160.0])
def test_meniscus_angle_reads_synthetic_arcs(theta):
    """The well-meniscus reader recovers the contact angle of an exact circular
    meniscus (tanh profile of width 1 across it) to 0.3 degrees, and reports
    whether the contact line is free or at a corner."""
    from well_angle import meniscus_angle
    nx, ny = 120, 90
    well = dict(x0=30, x1=90, y0=10, y1=70)
    a = (well["x1"] - well["x0"]) / 2.0
    xm = well["x0"] - 0.5 + a
    yc_line = 40.0  # contact-line height on both walls
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    if abs(theta - 90.0) < 1e-9:
        d = y - yc_line  # signed distance above the flat meniscus
    else:
        R = a / abs(np.cos(np.radians(theta)))
        # centre above the contact line when fluid 3 (below) wets (theta < 90)
        yc = yc_line + np.sign(90.0 - theta) * np.sqrt(R * R - a * a)
        rr = np.hypot(x - xm, y - yc)
        d = (R - rr) if theta < 90 else (rr - R)
    C3 = 0.5 * (1 - np.tanh(d / 2.0))
    got, heights, free = meniscus_angle(C3, well)
    assert got == pytest.approx(theta, abs=0.3)
    assert free
    assert heights[0] == pytest.approx(yc_line, abs=0.3) and heights[1] == pytest.approx(yc_line, abs=0.3)
    # the same meniscus with its contact line at the top corner is reported pinned
    pinned_well = dict(well, y1=int(yc_line + 1))
    assert not meniscus_angle(C3, pinned_well)[2]
