"""bench.py's host-side helpers, on the CPU: which blocks the oracle checks, and the compact record
of a workload line."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.argv = sys.argv[:1]
import bench  # noqa: E402


class _S:
    def __init__(self, N, overlap, nsamples):
        self.N, self.overlap, self.nsamples = N, overlap, nsamples


def test_small_workload_is_covered_whole_without_repeats():
    s = _S(256, 64, 1 << 16)                       # 342 blocks
    runs = bench.pick_runs([s], np.random.default_rng(0), 64, 4096)
    assert runs == [(0, b) for b in range(0, 342, 64)]


def test_large_workload_takes_first_last_and_seeded_runs():
    streams = [_S(1024, 256, 1 << 22) for _ in range(64)]   # 5462 blocks each
    runs = bench.pick_runs(streams, np.random.default_rng(12345), 64, 4096)
    assert len(runs) == 4096
    assert runs[0] == (0, 0)
    assert runs[1] == (63, 5462 - 64)                # the last stream's ragged end
    again = bench.pick_runs(streams, np.random.default_rng(12345), 64, 4096)
    assert runs == again                              # seeded
    for i, b0 in runs:
        assert 0 <= i < 64 and 0 <= b0 <= 5462 - 64


def test_brief_keeps_what_the_record_reports():
    line = {"config": {"workload": "w", "l2": "x"}, "value": 1.5, "unit": "Gsamples/s",
            "ms_per_step": 2.0, "steps": 3, "dtype": "f32",
            "roofline": {"frac": 0.5, "kernel": "k", "launch_ms": 2.0}, "gpu_launches": 3,
            "clocks": {"sm_mhz": 2070.0}, "rms_rel_err_sampled": 1e-7, "rms_tol": 2e-6,
            "cpu_baseline": {"samples": 10, "sample": "s", "value": 0.01, "cores": 16}}
    r = bench._brief(line)
    assert r["value"] == 1.5 and r["roofline_frac"] == 0.5 and r["rms_samples"] == 10
    assert r["clocks"] == {"sm_mhz": 2070.0} and r["cpu_cores"] == 16 and r["rms_tol"] == 2e-6


def test_profile_traffic_needs_matching_sources(tmp_path, monkeypatch):
    # a summary keyed to another source hash gives no traffic figure
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "k.md").write_text("source_hash: 000000000000\ndram_bytes_per_full_launch: 1e9\n")
    csrc = tmp_path / "paper_2406_14116_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in bench.KERNEL_SOURCES:
        (csrc / f).write_text("x")
    assert bench.profile_traffic("k") is None
    h = bench.source_hash()
    (tmp_path / "profiles" / "k.md").write_text(f"source_hash: {h}\ndram_bytes_per_full_launch: 1e9\n")
    assert bench.profile_traffic("k") == 1e9
