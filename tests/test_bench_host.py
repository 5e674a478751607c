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
