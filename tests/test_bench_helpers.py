"""The benchmark's profile bookkeeping (CPU): DRAM traffic and ncu issue
figures are reported from the committed profile summaries only while the
force kernel's sources still hash to the value the summary records, and the
traffic of workloads too large to capture scales with the cluster pairs."""
import os

import pytest

import bench


def _write(tmp, name, text):
    d = tmp / "profiles"
    d.mkdir(exist_ok=True)
    (d / name).write_text(text)


def test_traffic_and_counters_follow_the_source_hash(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "force_source_hash", lambda: "abc123")
    _write(tmp_path, "k_force8_w.md", "source-hash: abc123\ndram-bytes-per-launch: 1000\n"
                                      "issue-active-pct: 80.5\nfma-pipe-cycles-active-pct: 47.0\n"
                                      "fp32-lane-ops-pct: 42.0\ncounters-from: here\n")
    assert bench.profiled_traffic("w") == 1000.0
    c = bench.profiled_counters("w")
    assert c == {"issue_slots_busy_pct": 80.5, "fma_pipe_cycles_active_pct": 47.0,
                 "fp32_lane_ops_pct_of_issue_peak": 42.0, "profile": "here"}
    # the kernel changed since the capture: nothing is reported
    monkeypatch.setattr(bench, "force_source_hash", lambda: "def456")
    assert bench.profiled_traffic("w") is None
    assert bench.profiled_counters("w") is None
    # no summary for the workload
    assert bench.profiled_traffic("other") is None
    assert bench.profiled_counters("other") is None


def test_scaled_traffic_is_proportional_to_cluster_pairs(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "force_source_hash", lambda: "h")
    _write(tmp_path, "k_force8_water1m.md", "source-hash: h\ndram-bytes-per-launch: 2000\n"
                                            "cluster-pairs-per-launch: 100\n")
    assert bench.scaled_traffic(100) == pytest.approx(2000.0)
    assert bench.scaled_traffic(350) == pytest.approx(7000.0)
    monkeypatch.setattr(bench, "force_source_hash", lambda: "x")
    assert bench.scaled_traffic(350) is None


def test_force_source_hash_covers_the_force_kernel_files():
    h = bench.force_source_hash()
    assert len(h) == 12 and all(c in "0123456789abcdef" for c in h)
    for rel in bench.FORCE_SOURCES:
        assert os.path.exists(os.path.join(bench.ROOT, rel)), rel
