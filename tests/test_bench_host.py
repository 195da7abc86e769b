"""Host logic of bench.py that needs no GPU: the DRAM traffic record and its
source hash, the curve summary of the study modes, and the failure-stage
names against the C header."""
import os
import re

import pytest

import bench

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_traffic_record_matches_the_current_device_sources():
    """The committed record was taken on the sources as they are: its hash
    matches and every class the roofline can name has bytes per voxel."""
    bpv, note = bench.dram_bytes_per_voxel()
    assert note.startswith("ncu capture"), note
    for cls in ("x1_inv_matvec", "x1_fwd_tangent", "y_pass", "gamma_last_axis"):
        assert cls in bpv and 10.0 < bpv[cls] < 400.0, (cls, bpv.get(cls))


def test_traffic_record_is_dropped_when_the_hash_differs(tmp_path, monkeypatch):
    src = bench.TRAFFIC_FILE
    dst = tmp_path / "dram_bytes_per_voxel.txt"
    text = open(src).read()
    text = re.sub(r"kernel_sources_sha16 \S+", "kernel_sources_sha16 0000000000000000", text)
    dst.write_text(text)
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(dst))
    bpv, note = bench.dram_bytes_per_voxel()
    assert bpv == {} and "changed" in note
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.txt"))
    assert bench.dram_bytes_per_voxel() == ({}, "no traffic record")


def test_traffic_hash_covers_every_device_header():
    """A change to any listed source changes the hash (a kernel edit cannot
    keep a stale record alive)."""
    csrc = os.path.join(ROOT, "paper_2103_04770_gb300", "csrc")
    for f in bench.DEVICE_SOURCES:
        assert os.path.exists(os.path.join(csrc, f)), f
    for f in os.listdir(csrc):
        if f.endswith(".cuh"):
            assert f in bench.DEVICE_SOURCES, "device header %s not hashed" % f


def test_curve_summary_peak_and_ductility():
    # E11, S11, D_max, substeps
    pts = [[0.001, 50.0, 0.0, 1], [0.002, 100.0, 0.0, 1], [0.003, 120.0, 0.1, 1], [0.004, 110.0, 0.3, 1],
           [0.005, 95.0, 0.5, 2], [0.006, 90.0, 0.7, 1]]
    s = bench._curve_summary({"curve": pts})
    assert s["peak_S11"] == 120.0 and s["E11_at_peak"] == 0.003
    assert s["E11_at_80pct_past_peak"] == 0.005          # first point <= 96 past the peak
    assert s["last_E11"] == 0.006 and s["max_D"] == 0.7
    s = bench._curve_summary({"curve": pts[:4]})
    assert s["E11_at_80pct_past_peak"] is None
    assert bench._curve_summary({"curve": []}) == {}


def test_failure_stage_names_follow_the_header():
    h = open(os.path.join(ROOT, "include", "rve.h")).read()
    m = re.search(r"fail_stage;\s*/\*\s*on failure:(.*?)\*/", h, re.S)
    assert m, "fail_stage comment not found"
    doc = " ".join(m.group(1).split())
    for k, name in bench.FAIL_STAGES.items():
        if k == 0:
            assert "0 on success" in doc
            continue
        assert re.search(r"%d %s" % (k, name), doc, re.I), (k, name, doc)
