"""The bench line's measured DRAM traffic (host logic, no GPU): an ncu --csv
log of the brick kernels becomes one CSV row per kernel stamped with the
digest of the kernel's sources, and a row reads as measured only while that
digest matches the sources."""
from __future__ import annotations

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

HEADER = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size",'
          '"Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"')


def _row(i, kernel, metric, unit, value):
    return (f'"{i}","1","python3","h","{kernel}","1","13","(512, 1, 1)","(304, 1, 1)","0","10.3",'
            f'"Command line profiler metrics","{metric}","{unit}","{value}"')


def _log(tmp_path):
    k1 = "void k_brick_push_st<3, 1>(DevTree, BrickGeom, BrickPushArgs)"
    k2 = "void k_brick_pull_st<3>(DevTree, BrickGeom, BrickPullArgs)"
    other = "void k_scan_apply(const int *, long, int *)"
    lines = ["==PROF== Connected to process 1", HEADER,
             _row(0, k1, "dram__bytes_read.sum", "Gbyte", "3.25"),
             _row(0, k1, "dram__bytes_write.sum", "Mbyte", "1,500.5"),
             _row(0, k1, "gpu__time_duration.sum", "msecond", "1.5"),
             _row(1, other, "dram__bytes_read.sum", "byte", "999"),
             _row(2, k2, "dram__bytes_read.sum", "byte", "100"),
             _row(2, k2, "dram__bytes_write.sum", "byte", "50"),
             _row(2, k2, "gpu__time_duration.sum", "usecond", "20"),
             _row(3, k2, "dram__bytes_read.sum", "byte", "300"),
             _row(3, k2, "dram__bytes_write.sum", "byte", "150"),
             _row(3, k2, "gpu__time_duration.sum", "nsecond", "40000"),
             "==PROF== Disconnected from process 1"]
    p = tmp_path / "dram.csv"
    p.write_text("\n".join(lines) + "\n")
    return p


def _rows(text):
    import csv
    return {r["kernel"]: r for r in csv.DictReader(ln for ln in text.splitlines() if not ln.startswith("#"))}


def test_ingest_sums_each_kernel_and_stamps_its_sources(tmp_path):
    rows = _rows(bench.ingest_ncu(str(_log(tmp_path)), "langmuir3d", 1000))
    assert set(rows) == {"k_brick_push_st", "k_brick_pull_st"}   # other kernels are left out
    k1, k2 = rows["k_brick_push_st"], rows["k_brick_pull_st"]
    assert (k1["launches"], k1["read_bytes"], k1["write_bytes"], k1["duration_ns"]) == \
        ("1", "3250000000", "1500500000", "1500000")
    assert (k2["launches"], k2["read_bytes"], k2["write_bytes"], k2["duration_ns"]) == \
        ("2", "400", "200", "60000")
    assert k1["particles"] == "1000" and k1["workload"] == "langmuir3d"
    assert k1["sources_digest"] == bench.kernel_digest("k_brick_push_st")


def test_traffic_reads_as_measured_only_for_the_current_sources(tmp_path, monkeypatch):
    text = bench.ingest_ncu(str(_log(tmp_path)), "langmuir3d", 1000)
    # the pull row as if captured from other sources (both brick kernels share theirs)
    lines = [ln.rsplit(",", 1)[0] + "," + "0" * 16 if ",k_brick_pull_st," in ln else ln for ln in text.splitlines()]
    csv_path = tmp_path / "traffic.csv"
    csv_path.write_text("\n".join(lines) + "\n")
    monkeypatch.setattr(bench, "TRAFFIC_CSV", str(csv_path))
    per_launch, row = bench.measured_traffic("langmuir3d", "k_brick_push_st")
    assert per_launch == pytest.approx(3250000000 + 1500500000) and row["kernel"] == "k_brick_push_st"
    per_launch, row = bench.measured_traffic("langmuir3d", "k_brick_pull_st")
    assert per_launch is None and row is not None          # captured from other sources: unmeasured
    assert bench.measured_traffic("twostream3d", "k_brick_push_st") == (None, None)
    monkeypatch.setattr(bench, "TRAFFIC_CSV", str(tmp_path / "missing.csv"))
    assert bench.measured_traffic("langmuir3d", "k_brick_push_st") == (None, None)


def test_digest_follows_every_source_file(tmp_path, monkeypatch):
    a, b = tmp_path / "a.cu", tmp_path / "b.cuh"
    a.write_text("kernel A\n")
    b.write_text("header B\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setitem(bench.KERNEL_SOURCES, "k_test", ("a.cu", "b.cuh"))
    d0 = bench.kernel_digest("k_test")
    b.write_text("header B, one comment more\n")
    assert bench.kernel_digest("k_test") != d0
    b.write_text("header B\n")
    assert bench.kernel_digest("k_test") == d0
