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


def _sampler(**attrs):
    s = object.__new__(bench.ClockSampler)
    s.proc = s.path = s.thread = s.nvml = s.handle = None
    s.samples = []
    for k, v in attrs.items():
        setattr(s, k, v)
    return s


def test_clock_sampler_nvml_summary():
    """NVML samples (SM MHz, clock-event-reason bits) reduce to the median
    clock, the maximum clock NVML reports and the named reasons seen."""
    import threading

    class FakeNvml:
        def nvmlDeviceGetMaxClockInfo(self, handle, kind, out):
            assert kind == 1                       # SM clock domain
            out._obj.value = 2070
            return 0

    t = threading.Thread(target=lambda: None)
    t.start()
    s = _sampler(nvml=FakeNvml(), thread=t, samples=[(2070, 0x4), (2055, 0x0), (2070, 0x8 | 0x4)])
    out = s.stop()
    assert out == {"sm_mhz": 2070, "sm_max_mhz": 2070, "reasons": ["hw_slowdown", "sw_power_cap"],
                   "samples": 3, "source": "nvml"}


def test_clock_sampler_nvidia_smi_summary(tmp_path):
    """The nvidia-smi fallback: CSV rows of the query, reasons named where
    their column says Active."""
    class FakeProc:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    path = tmp_path / "clocks.csv"
    path.write_text("0, 2070, 2070, 910.2, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n"
                    "0, 1980, 2070, 1390.0, 0x0000000000000044, Not Active, Active, Not Active, Active\n"
                    "0, 2070, 2070, 905.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
                    "garbage line\n")
    s = _sampler(proc=FakeProc(), path=str(path))
    out = s.stop()
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["hw_thermal_slowdown", "sw_power_cap"],
                   "samples": 3, "source": "nvidia-smi"}
    assert not path.exists()


def test_clock_sampler_without_a_source():
    assert _sampler().stop() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
