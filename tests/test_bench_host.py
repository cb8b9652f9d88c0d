"""Host-side bookkeeping of bench.py (no GPU): the recorded DRAM traffic of the
thread-per-merge kernel is reported only for the workload and sources it was
captured on, and the algorithmic bytes follow the per-level formula."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_only_for_the_captured_workload():
    t = bench.kernel_traffic()
    if bench.KERNEL_TRAFFIC["sources_sha256"] == bench.sources_sha256():
        assert t == bench.KERNEL_TRAFFIC["bytes_per_launch"]
    else:
        assert t is None
    assert bench.kernel_traffic(1 << 22) is None
    assert bench.kernel_traffic(1 << 24, ("cube",)) is None
    assert bench.kernel_traffic(1 << 24, bench.DISTS, default_plan=False) is None


def test_traffic_dropped_when_the_sources_change(monkeypatch):
    monkeypatch.setitem(bench.KERNEL_TRAFFIC, "sources_sha256", "0" * 64)
    assert bench.kernel_traffic() is None


def test_issue_roofline_from_the_recorded_counts():
    sha_ok = bench.KERNEL_ISSUE["sources_sha256"] == bench.sources_sha256()
    r = bench.kernel_issue(4.0, 152, 2000.0)
    if not sha_ok:
        assert r is None
        return
    w = bench.KERNEL_ISSUE["warp_inst_per_launch"]
    assert r["bound"] == "alu" and r["unit"] == "Gwarp-inst/s"
    assert abs(r["achieved"] - w / 4e-3 / 1e9) < 1e-6
    assert abs(r["peak"] - 4 * 152 * 2.0) < 1e-9
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    assert 1.0 <= r["active_lanes_per_inst"] <= 32.0
    assert bench.kernel_issue(4.0, 152, 2000.0, 1 << 22) is None
    assert bench.kernel_issue(4.0, 152, 2000.0, default_plan=False) is None
    assert bench.kernel_issue(0.0, 152, 2000.0) is None


def test_batched_oracle_baseline_on_a_small_batch():
    from paper_1205_1171_gb300 import inputs

    xyz, off, _ = inputs.batch(96, inputs.seed_for(4))
    r = bench.batched_cpu_baseline(xyz, off, sample=64, workers=2)
    assert "unavailable" not in r, r
    assert r["cores"] == 2 and r["kind"] == "oracle" and r["hulls_per_s"] > 0
    assert r["sample"].startswith("first 64 clouds")
