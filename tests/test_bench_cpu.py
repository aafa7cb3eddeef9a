"""Host-side pieces of bench.py that shape its JSON line (CPU only)."""
from __future__ import annotations

import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_roofline_of_picks_the_dominant_class():
    prof = {"onesweep": {"launches": 10, "ms": 4.0, "bytes": 8.0e9},
            "rerank": {"launches": 5, "ms": 1.0, "bytes": 1.0e9}}
    roof, kernels = bench.roofline_of(prof, 4000.0, "measured", steps=2)
    assert roof["kernel"] == "onesweep"
    assert abs(roof["achieved"] - 2000.0) < 1e-9          # 8 GB in 4 ms
    assert abs(roof["frac"] - 0.5) < 1e-12
    assert roof["bound"] == "hbm" and roof["unit"] == "GB/s"
    assert abs(kernels["onesweep"]["ms_per_step"] - 2.0) < 1e-12
    assert abs(sum(k["share"] for k in kernels.values()) - 1.0) < 1e-12


def test_roofline_of_without_profile():
    assert bench.roofline_of({}, 1.0, "measured", steps=1) == (None, {})


def test_pctl():
    xs = [5, 1, 4, 2, 3]
    assert bench.pctl(xs, 50) == 3
    assert bench.pctl(xs, 0) == 1 and bench.pctl(xs, 100) == 5
    assert bench.pctl([], 50) is None


class _FakeProc:
    def __init__(self, out):
        self.out = out

    def terminate(self):
        pass

    def kill(self):
        pass

    def communicate(self, timeout=None):
        return self.out, ""


def test_clock_sampler_parses_median_and_reasons():
    rows = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2050, 2070, 950.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 960.3, 0x0, Not Active, Not Active, Not Active, Not Active",
            "garbage line"]
    cs = bench.ClockSampler(0)
    cs.proc = _FakeProc("\n".join(rows))
    got = cs.stop()
    assert got["sm_mhz"] == 2070.0 and got["sm_max_mhz"] == 2070.0 and got["samples"] == 3
    assert got["reasons"] == ["sw_power_cap"]


def test_clock_sampler_without_nvidia_smi():
    cs = bench.ClockSampler(0)
    assert cs.stop() is None


def test_measured_peak_reads_the_peaks_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peak() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6683.8}))
    assert bench.measured_peak() == (6683.8, "measured")


def test_dist_env_defaults(monkeypatch):
    for k in ("RANK", "LOCAL_RANK", "WORLD_SIZE"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (0, 0, 1)


def test_traffic_ratio_only_for_the_captured_source(tmp_path, monkeypatch):
    """A DRAM-per-algorithmic-byte ratio is reported only while the kernel source
    hashes to the one the counters were taken on."""
    import hashlib

    src = tmp_path / "k.cu"
    src.write_text("kernel v1\n")
    prof = tmp_path / "profiles"
    prof.mkdir()
    good = hashlib.sha1(src.read_bytes()).hexdigest()
    (prof / "traffic.json").write_text(json.dumps({
        "onesweep": {"dram_per_algorithmic_byte": 0.9, "valid": True, "source": "k.cu", "source_sha1": good},
        "rerank": {"dram_per_algorithmic_byte": 1.1, "valid": True, "source": "k.cu", "source_sha1": "0" * 40},
        "lcp": {"dram_per_algorithmic_byte": 1.0, "valid": False, "source": "k.cu", "source_sha1": good}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_ratio("onesweep") == 0.9
    assert bench.traffic_ratio("rerank") is None      # source changed since the capture
    assert bench.traffic_ratio("lcp") is None         # marked invalid
    assert bench.traffic_ratio("segsort") is None     # never captured
    src.write_text("kernel v2\n")
    assert bench.traffic_ratio("onesweep") is None
