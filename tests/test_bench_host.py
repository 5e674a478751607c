"""Host-side logic of bench.py, on CPU: the clock record parsed from nvidia-smi lines
(throttle reasons, malformed lines), the DRAM-traffic record that is reported only
while the kernel's source is the one it was taken on, and the choice of extra legs."""
from __future__ import annotations

import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    return bench


def test_clock_samples_median_and_reasons():
    b = _bench()
    text = "\n".join([
        "0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1995, 2070, 1380.2, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2055, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ])
    c = b.parse_clock_samples(text)
    assert c == dict(sm_mhz=2055.0, sm_max_mhz=2070.0, reasons=["sw_power_cap"], samples=3)


def test_clock_samples_report_thermal_and_hardware_slowdowns():
    b = _bench()
    text = ("0, 1500, 2070, 1400, 0x48, Active, Not Active, Active, Not Active\n"
            "0, 1400, 2070, 1400, 0x48, Not Active, Active, Not Active, Not Active\n")
    c = b.parse_clock_samples(text)
    assert c["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert c["sm_mhz"] == 1450.0


def test_clock_samples_empty():
    assert _bench().parse_clock_samples("") is None
    assert _bench().parse_clock_samples("no gpu here\n") is None


def test_traffic_record_follows_the_kernel_source(tmp_path, monkeypatch):
    b = _bench()
    csrc = tmp_path / "paper_2512_01251_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (csrc / "k.cu").write_text("__global__ void k() {}\n")
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    rec = dict(bytes_per_launch=123, source_hash=b.source_hash("k.cu"))
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"k": rec}))
    assert b.measured_traffic("k", ["k.cu"])["bytes_per_launch"] == 123
    assert b.measured_traffic("other", ["k.cu"]) is None
    (csrc / "k.cu").write_text("__global__ void k() { /* changed */ }\n")
    assert b.measured_traffic("k", ["k.cu"]) is None


def test_leg_selection(monkeypatch):
    b = _bench()
    monkeypatch.setattr(sys, "argv", ["bench.py", "--legs", "batched,replay"])
    a = b.parse()
    assert a.legs == "batched,replay" and a.steps == 10 and a.warmup == 3 and a.gpus == 1
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    assert b.parse().legs == "all"


def test_oracle_slabs_partition_the_workload():
    """The reference arm's layer samples: slabs of root-block layers covering the domain
    add up to exactly the units of the whole workload."""
    b = _bench()
    from oracle import oracle as O
    from synth import workload
    w = workload("star_20k")
    v, t = w.build_mesh()
    full, _ = b.oracle_lines_full(v, t, w, 27)
    tri9 = O.tri_coords(O.int_coords(v, w.R), t)
    parts = sum(b.oracle_slab(tri9, w, 27, z0, z0 + 3)[0] for z0 in range(0, w.R, 3))
    assert parts == full


def test_step_roofline_sums_the_calls():
    b = _bench()
    med = {"mesh": 0.3, "bin0": 0.5, "bin1": 1.0, "voxelize0": 0.1, "voxelize1": 0.2, "refine_flags0": 0.4,
           "forest_refine0": 0.1, "cutlinks_prep": 0.5, "cutlinks_emit": 4.0}
    r = b.step_roofline(med, 1000, [8, 64], [(500, 0), (400, 3000)], 20000, 10 ** 9, 6000.0, 40.0, 8.0, 6.0)
    assert set(r["per_call"]) == {"mesh", "bin0", "bin1", "voxelize0", "voxelize1", "refine_flags0", "forest_refine0",
                                  "cutlinks"}
    lk = r["per_call"]["cutlinks"]
    assert lk["bound"] == "alu" and abs(lk["roof_ms"] - (10 ** 9 * 48 + 20000 * 60) / 40e12 * 1e3) < 1e-3
    assert abs(r["step_roof_ms"] - sum(x["roof_ms"] for x in r["per_call"].values())) < 1e-3
    assert abs(r["step_frac"] - r["step_roof_ms"] / 8.0) < 1e-3 and abs(r["replay_frac"] - r["step_roof_ms"] / 6.0) < 1e-3
    assert abs(lk["ms"] - 4.5) < 1e-9  # link preparation plus the table
    # the link table's bytes count the records of the finest bins' distinct triangles
    by = 27 * 8 * 64 + 4 * 3000 + 13 * 20000
    assert lk["bytes"] == by + 48 * 400
    r2 = b.step_roofline(med, 1000, [8, 64], [(500, 0), (400, 3000)], 20000, 10 ** 9, 6000.0, 40.0, 8.0, 6.0,
                         link_tris=900)
    assert r2["per_call"]["cutlinks"]["bytes"] == by + 48 * 900
