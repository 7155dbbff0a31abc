"""Host logic of bench.py that needs no GPU: the measured-traffic record (it is
reported only while the digest of the listed sources still matches), the
clock sampler's selection of the samples inside the timed region, and the
choice of arrays the end-to-end step copies from the host."""
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


class _Layout:
    """The attributes of a slice layout that the end-to-end copies use."""

    def __init__(self, mode, N, nnz, nfibers=None):
        import torch
        self.mode = mode
        self.nnz = nnz
        self.idx = [torch.arange(nnz, dtype=torch.int32) + 100 * k for k in range(N)]
        self.val = torch.rand(nnz)
        self.row_ptr = torch.arange(nnz + 1, dtype=torch.int32)
        self.nfibers = nfibers or 0
        if nfibers is None:
            self.fid = self.fcoord = None
        else:
            self.fid = torch.zeros(nnz, dtype=torch.int32)
            self.fcoord = [None if k == mode else torch.arange(nnz, dtype=torch.int32)
                           for k in range(N)]


def _inputs(layouts, N):
    import torch
    return {"slices": layouts, "tidx": [torch.zeros(5, dtype=torch.int32) for _ in range(N)],
            "tval": torch.zeros(5), "ready": None}


def test_e2e_ships_compact_layouts():
    """A mode with fibers ships values, row_ptr, fid and nfibers entries of its
    fiber coordinates (no coordinate arrays: the step rebuilds them); a mode
    without fibers ships the other modes' coordinates too; never the own
    mode's coordinates; the test set is the last group."""
    N, nnz = 3, 40
    lays = [_Layout(0, N, nnz, nfibers=7), _Layout(1, N, nnz), _Layout(2, N, nnz, nfibers=9)]
    inp = _inputs(lays, N)
    groups = bench.e2e_groups(inp, N)
    assert len(groups) == N + 1
    g0 = groups[0]
    assert g0[0] is lays[0].val and g0[1] is lays[0].row_ptr and g0[2] is lays[0].fid
    assert [t.numel() for t in g0[3:]] == [7, 7] and len(g0) == 5
    g1 = groups[1]
    assert g1[0] is lays[1].idx[0] and g1[1] is lays[1].idx[2]
    assert g1[2] is lays[1].val and g1[3] is lays[1].row_ptr and len(g1) == 4
    assert [t.numel() for t in groups[2][3:]] == [9, 9]
    for g, sl in zip(groups, lays):
        assert all(t is not sl.idx[sl.mode] for t in g)
    assert groups[N][-1] is inp["tval"] and len(groups[N]) == N + 1


def test_e2e_second_set_owns_its_buffers():
    """The second buffer set has fresh tensors of the same shapes for every
    shipped or rebuilt array, and shares nothing written by a step's copies."""
    N, nnz = 3, 40
    lays = [_Layout(0, N, nnz, nfibers=7), _Layout(1, N, nnz), _Layout(2, N, nnz, nfibers=9)]
    inp = _inputs(lays, N)
    two = bench.e2e_clone_set(inp)
    ga, gb = bench.e2e_groups(inp, N), bench.e2e_groups(two, N)
    assert [[tuple(t.shape) for t in g] for g in ga] == [[tuple(t.shape) for t in g] for g in gb]
    for x, y in zip(ga, gb):
        for a, b in zip(x, y):
            assert a.data_ptr() != b.data_ptr()
    for a, b in zip(lays, two["slices"]):
        assert b.mode == a.mode and b.nfibers == a.nfibers
        assert all(p.data_ptr() != q.data_ptr() for p, q in zip(a.idx, b.idx))
