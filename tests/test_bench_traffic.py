"""The roofline's `traffic` figure: bench.py reads the DRAM bytes per search
launch from the committed ncu summary only while that summary was taken on
the current search kernel source (a recorded hash), so a kernel edited
since the capture reports null instead of a stale figure."""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _summary(tmp_path, sha, nbytes="4.9065e9", workload="paper_24x24_15k"):
    p = tmp_path / f"k_screen_{workload}.txt"
    p.write_text("# header line: with a colon\n"
                 f"dram_bytes_per_launch: {nbytes}\n"
                 f"source_sha256: {sha}\n")
    return str(tmp_path)


def test_committed_summary_is_plausible():
    # a summary taken on the kernel as it stands: its bytes are the table's
    # (no re-reads); after a kernel edit the figure is null until re-captured
    t = bench._traffic()
    if t is None:
        pytest.skip("the committed summary predates the current search source")
    algorithmic = 2.0 * 162336 * 15000
    assert 1.0 <= t / algorithmic < 1.02  # row padding to 256 entries


def test_traffic_is_read_for_the_current_source(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "PROFILE_DIR", _summary(tmp_path, bench.search_source_digest()))
    assert bench._traffic() == 4.9065e9


def test_traffic_is_only_the_profiled_workloads(tmp_path, monkeypatch):
    # a summary of the 24x24 / 15k table says nothing about another workload's
    monkeypatch.setattr(bench, "PROFILE_DIR", _summary(tmp_path, bench.search_source_digest()))
    assert bench._traffic("search_16x16_15k") is None


def test_traffic_is_null_once_the_kernel_changed(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "PROFILE_DIR", _summary(tmp_path, "0" * 64))
    assert bench._traffic() is None


def test_traffic_is_null_without_a_summary(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "PROFILE_DIR", str(tmp_path / "missing"))
    assert bench._traffic() is None


def test_cpu_model_is_named():
    # the CPU baseline names the host CPU beside its thread count
    m = bench.cpu_model()
    assert isinstance(m, str) and m and m != "unknown"
