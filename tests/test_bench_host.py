"""Host-side bookkeeping of bench.py (no GPU): the recorded DRAM traffic of the
thread-per-merge kernel is reported only for the workload and sources it was
captured on, and the algorithmic bytes follow the per-level formula."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_only_for_the_captured_workload_and_plan():
    t = bench.kernel_traffic()
    if bench.KERNEL_TRAFFIC["sources_sha256"] == bench.sources_sha256():
        assert t == bench.KERNEL_TRAFFIC["bytes_per_launch"]
    else:
        assert t is None
    assert bench.kernel_traffic(1 << 22) is None
    assert bench.kernel_traffic(1 << 24, ("cube",)) is None
    assert bench.kernel_traffic(1 << 24, bench.DISTS, {}) is None  # another plan
    assert bench.kernel_traffic(1 << 24, bench.DISTS, dict(bench.KERNEL_KNOBS, cmp_level=9)) is None


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
    assert bench.kernel_issue(4.0, 152, 2000.0, knobs={}) is None
    assert bench.kernel_issue(0.0, 152, 2000.0) is None


def test_the_recorded_knobs_are_the_shipped_tuned_plan():
    from paper_1205_1171_gb300 import autotune

    assert autotune.lookup("NVIDIA GB300", 1 << 24, path=None, cls="volume") == bench.KERNEL_KNOBS


def test_batched_oracle_baseline_on_a_small_batch():
    from paper_1205_1171_gb300 import inputs

    xyz, off, _ = inputs.batch(96, inputs.seed_for(4))
    r, digests = bench.batched_cpu_baseline(xyz, off, sample=64, workers=2)
    assert "unavailable" not in r, r
    assert r["cores"] == 2 and r["kind"] == "oracle" and r["hulls_per_s"] > 0
    assert r["sample"].startswith("first 64 clouds")
    assert sorted(digests) == list(range(64))
    r, digests = bench.batched_cpu_baseline(xyz, off, sample=32, workers=2, every_cloud=True)
    assert r["sample"].startswith("first 32 clouds")  # the timed part
    assert sorted(digests) == list(range(96))  # every cloud digested for the parity check


def test_batch_parity_accepts_the_oracle_faces_and_rejects_a_changed_face():
    import numpy as np
    import pytest
    import torch

    import oracle
    from paper_1205_1171_gb300 import inputs

    xyz, off, _ = inputs.batch(12, inputs.seed_for(4))
    sizes = np.diff(off)
    foff = np.zeros(len(off), np.int64)
    foff[1:] = np.cumsum(np.where(sizes >= 3, 2 * sizes - 4, 0))
    faces = np.full((int(foff[-1]), 3), -1, np.int32)
    nf = np.zeros(12, np.int64)
    digests = {}
    for b in range(12):  # a batch output laid out as the GPU writes it, here from the oracle
        f = oracle.hull(xyz[off[b]: off[b + 1]])
        faces[foff[b]: foff[b] + len(f)] = f
        nf[b] = len(f)
        digests[b] = (len(f), bench.face_digest(f))
    ft, nt = torch.from_numpy(faces), torch.from_numpy(nf)
    assert bench.batch_parity(ft, nt, foff, digests) == {"clouds": 12, "bit_exact": True}
    faces[foff[5] + 1, [1, 2]] = faces[foff[5] + 1, [2, 1]]  # one face turned inside out
    with pytest.raises(RuntimeError, match="cloud 5"):
        bench.batch_parity(torch.from_numpy(faces), nt, foff, digests)
    assert bench.batch_parity(ft, nt, foff, {}) == {"clouds": 0, "bit_exact": None}


def test_batch_counts_scale_with_the_clouds_and_need_the_recorded_knobs():
    ok = bench.BATCH_COUNTS["sources_sha256"] == bench.sources_sha256(bench.BATCH_SOURCES)
    c = bench.batch_counts(bench.BATCH_COUNTS["knobs"], 4 * bench.BATCH_COUNTS["clouds"])
    if not ok:
        assert c is None
        return
    assert c["warp_inst"] == 4 * bench.BATCH_COUNTS["warp_inst"]
    assert c["dram_bytes"] == 4 * bench.BATCH_COUNTS["dram_bytes"]
    assert 1.0 <= c["active_lanes_per_inst"] <= 32.0
    assert bench.batch_counts({"batch_warp_nodes": 64}, 65536) is None
