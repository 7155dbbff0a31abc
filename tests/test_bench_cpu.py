"""Host logic of bench.py that needs no GPU: the measured-traffic record (it is
reported only while the digest of the listed sources still matches) and the
clock sampler's selection of the samples inside the timed region."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _record(tmp_path, sources, digest, nbytes=1234.0, key="w|fp32|slices|factor"):
    p = tmp_path / "traffic.json"
    p.write_text(json.dumps({key: {"bytes_per_launch": nbytes, "sources": sources,
                                   "digest": digest}}))
    return str(p)


def test_traffic_reported_while_sources_match(tmp_path, monkeypatch):
    sources = ["bench.py", "README.md"]
    path = _record(tmp_path, sources, bench.source_digest(sources))
    monkeypatch.setattr(bench, "TRAFFIC_PATH", path)
    assert bench.measured_traffic("w|fp32|slices|factor") == 1234.0
    assert bench.measured_traffic("other|fp32|slices|factor") is None


def test_traffic_withheld_after_a_source_changes(tmp_path, monkeypatch):
    src = tmp_path / "kernel.cu"
    src.write_text("kernel v1\n")
    rel = os.path.relpath(str(src), ROOT)
    path = _record(tmp_path, [rel], bench.source_digest([rel]))
    monkeypatch.setattr(bench, "TRAFFIC_PATH", path)
    assert bench.measured_traffic("w|fp32|slices|factor") == 1234.0
    src.write_text("kernel v2\n")
    assert bench.measured_traffic("w|fp32|slices|factor") is None


def test_traffic_missing_or_malformed_record(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "TRAFFIC_PATH", str(tmp_path / "absent.json"))
    assert bench.measured_traffic("w|fp32|slices|factor") is None
    bad = tmp_path / "bad.json"
    bad.write_text("{not json")
    monkeypatch.setattr(bench, "TRAFFIC_PATH", str(bad))
    assert bench.measured_traffic("w|fp32|slices|factor") is None


def test_digest_depends_on_names_and_contents(tmp_path):
    a = tmp_path / "a.txt"
    b = tmp_path / "b.txt"
    a.write_text("x")
    b.write_text("x")
    ra, rb = (os.path.relpath(str(p), ROOT) for p in (a, b))
    assert bench.source_digest([ra]) != bench.source_digest([rb])  # same bytes, other file
    assert bench.source_digest([ra, rb]) != bench.source_digest([rb, ra])  # order counts


def test_clock_sampler_keeps_samples_of_the_timed_region():
    c = bench.ClockSampler(0)
    c.t0, c.t1 = 100.0, 101.0
    line = "0, {sm}, 2070, 900.0, 0x0, Not Active, Not Active, {th}, Active"
    c.lines = [(99.0, line.format(sm=1000, th="Not Active")),     # before the region
               (100.2, line.format(sm=2070, th="Not Active")),
               (100.9, line.format(sm=2060, th="Active")),
               (101.05, line.format(sm=2070, th="Not Active")),   # covers the end
               (102.0, line.format(sm=500, th="Not Active"))]     # after the region
    s = c.summary()
    assert s["samples"] == 3
    assert s["sm_mhz"] == 2070.0
    assert s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap", "sw_thermal_slowdown"]


def test_clock_sampler_without_nvidia_smi(monkeypatch):
    def missing(*a, **k):
        raise FileNotFoundError("nvidia-smi")
    monkeypatch.setattr(bench.subprocess, "Popen", missing)
    with bench.ClockSampler(0) as c:
        pass
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
