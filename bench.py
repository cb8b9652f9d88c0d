"""Benchmark of the GB300 kinetic divide-and-conquer 3D hull.

One step = the whole hot path (range check, radix sort, every merge level of
both passes, face emission and canonical sort) over the two n = 2^24 clouds of
the headline workload: uniform in the cube [-2^20, 2^20)^3 and an isotropic
Gaussian (sigma = 2^18) clipped to the cube.  Points are already resident in
HBM when the timed region starts (each cloud is 201 MB, above the 129 MB L2).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the plain serial implementation the
CUDA path is checked against) on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpoints/s per hull at n=2^24 and hulls/s batched (bit-exact), % of HBM roofline"
UNIT = "Mpoints/s"
N_POINTS = 1 << 24
DISTS = ("cube", "gauss")
WORKLOAD = "single hulls at n=2^24: uniform cube + isotropic Gaussian sigma=2^18 clipped to the cube (one of each per step)"
ORACLE_SAMPLE = 1 << 17  # points per cloud in one step of the reference arm
BASELINE_SAMPLE = 1 << 19  # points per cloud in the cpu_baseline leg


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# DRAM bytes (read + write) and instructions per launch of the thread-per-merge
# level kernel (levels 3-11 of the two n = 2^24 clouds, 18 launches, averaged),
# from one-pass ncu captures of `bench.py --profile-once` (the command and the
# per-level figures are in profiles/), valid for the merge sources whose SHA-256
# and the plan knobs that are recorded with them.  The instruction counts give
# the second roofline: instruction issue, against 4 warp instructions per SM
# per cycle (one per SM sub-partition).
KERNEL_SOURCES_SHA = "f23555662a8a0d1d15883a65d3c4324d3907c14d68a693f6d8a5b078f1c8ded2"
# (the shortest time window, seg_events_min, acts only from the first time-window
# level, 12, above every level the counted kernel runs, 3-11)
KERNEL_KNOBS = {"cmp_level": 12, "level_occupancy": 0, "seg_events": 256, "seg_level": 12, "seg_min_events": 0,
                "seg_events_min": 64}
KERNEL_TRAFFIC = {"bytes_per_launch": 2578944028, "sources_sha256": KERNEL_SOURCES_SHA, "knobs": KERNEL_KNOBS}
TRAFFIC_SOURCES = ("paper_1205_1171_gb300/csrc/merge.cu", "paper_1205_1171_gb300/csrc/merge.cuh",
                   "paper_1205_1171_gb300/csrc/predicates.cuh")
KERNEL_ISSUE = {"warp_inst_per_launch": 1523402311, "thread_inst_per_launch": 18230573092,
                "sources_sha256": KERNEL_SOURCES_SHA, "knobs": KERNEL_KNOBS}
ISSUE_PER_SM_PER_CYCLE = 4
# The batch kernel on the first 4096 clouds of the batch's draw (its four
# size-class launches, the tuned cut-over), from one ncu capture of
# `bench.py --batch-only 4096`: DRAM bytes and instructions per cloud, valid
# for the batch sources and knobs recorded with them; the 65,536-cloud batch
# is the same draw, so its counts scale with the clouds.
BATCH_SOURCES = ("paper_1205_1171_gb300/csrc/batch.cu", "paper_1205_1171_gb300/csrc/merge.cuh",
                 "paper_1205_1171_gb300/csrc/predicates.cuh")
BATCH_COUNTS = {"clouds": 4096, "dram_bytes": 60569088, "warp_inst": 7648474235, "thread_inst": 124714875403,
                "knobs": {"batch_warp_nodes": 16},
                "sources_sha256": "0e8bd20198bf60be29fc0f2d9584b43395aab8b702099997ccb5804485af05a0"}


def sources_sha256(files=None) -> str:
    import hashlib

    h = hashlib.sha256()
    for rel in files or TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _recorded_applies(rec, npts, dists, knobs) -> bool:
    return (bool(rec) and npts == 1 << 24 and tuple(dists) == tuple(DISTS) and knobs == rec["knobs"]
            and rec["sources_sha256"] == sources_sha256())


def kernel_traffic(npts: int = 1 << 24, dists=DISTS, knobs=None):
    """The recorded DRAM traffic per launch: None once the kernel changed, and
    None for any other workload or plan knobs than the ones it was captured on."""
    knobs = KERNEL_KNOBS if knobs is None else knobs
    return KERNEL_TRAFFIC["bytes_per_launch"] if _recorded_applies(KERNEL_TRAFFIC, npts, dists, knobs) else None


def kernel_issue(ms_per_launch: float, sms: int, sm_mhz: float, npts: int = 1 << 24, dists=DISTS, knobs=None):
    """The instruction-issue roofline of the thread-per-merge kernel from the
    recorded instruction counts and the live launch time, or None where the
    counts do not apply (other workload, plan knobs or sources)."""
    knobs = KERNEL_KNOBS if knobs is None else knobs
    if not _recorded_applies(KERNEL_ISSUE, npts, dists, knobs) or ms_per_launch <= 0:
        return None
    w = KERNEL_ISSUE["warp_inst_per_launch"]
    achieved = w / (ms_per_launch / 1e3) / 1e9
    peak = ISSUE_PER_SM_PER_CYCLE * sms * sm_mhz / 1e3
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gwarp-inst/s", "frac": achieved / peak,
            "warp_inst_per_launch": w,
            "active_lanes_per_inst": KERNEL_ISSUE["thread_inst_per_launch"] / w,
            "peak_basis": f"{ISSUE_PER_SM_PER_CYCLE} warp instructions per SM per cycle x {sms} SMs x "
                          f"{sm_mhz:.0f} MHz (median SM clock of the timed region)"}


def batch_counts(knobs, clouds: int):
    """The recorded batch-kernel counts scaled to `clouds` clouds of the same
    draw, or None where they do not apply (other knobs or sources)."""
    rec = BATCH_COUNTS
    if knobs != rec["knobs"] or rec["sources_sha256"] != sources_sha256(BATCH_SOURCES):
        return None
    f = clouds / rec["clouds"]
    return {"dram_bytes": rec["dram_bytes"] * f, "warp_inst": rec["warp_inst"] * f,
            "active_lanes_per_inst": rec["thread_inst"] / rec["warp_inst"]}


def max_over_ranks(x: float, dist, device: str = "cuda") -> float:
    """The largest x over the ranks (every rank gets it); x itself without a process group."""
    if not dist:
        return x
    import torch

    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_inputs(rank: int, n: int = N_POINTS, dists=DISTS):
    from paper_1205_1171_gb300 import inputs

    return [inputs.cloud_seeded(d, n, inputs.seed_for(30 + i) + 1000 * rank) for i, d in enumerate(dists)]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def level_alg_bytes(n: int, ev: np.ndarray, level: int) -> int:
    """Algorithmic bytes of merge level `level`, both passes: 4 B per child and
    per parent event (an event is one int32 rank) and 12 B per point whose
    coordinates the merges read.  Those points are the child event points and
    the four x-extremes of each merge, so E(level - 1) + 4 M bounds them."""
    half = 1 << (level - 1)
    merges = (n >> level) + (1 if n % (1 << level) > half else 0)
    return sum(4 * (int(ev[p, level - 1]) + int(ev[p, level])) + 12 * (int(ev[p, level - 1]) + 4 * merges)
               for p in range(2))


def alg_bytes(n: int, ev: np.ndarray, fused_l1: int, nfaces: int, seg_level: int) -> dict:
    """Algorithmic bytes per call and phase: read the input (12 n) and write the
    sorted points (16 n); the merge levels; 12 B per output face."""
    L = int(np.ceil(np.log2(n)))
    l1 = min(fused_l1, L)
    out = {"sort": 28 * n, "fused": 0, "levels": 0, "seg": 0, "faces": 12 * nfaces}
    for lv in range(2, L + 1):
        phase = "fused" if lv <= l1 else ("seg" if lv >= seg_level else "levels")
        out[phase] += level_alg_bytes(n, ev, lv)
    return out


def run_reference(args, rank: int, world: int):
    """The CPU oracle, as it stands, on bounded samples of the same workload."""
    if rank != 0:
        return
    import oracle

    oracle.build()
    clouds = make_inputs(0)
    samples = [c[:ORACLE_SAMPLE].copy() for c in clouds]
    for _ in range(args.warmup):
        for s in samples:
            oracle.hull(s)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for s in samples:
            oracle.hull(s)
    dt = time.perf_counter() - t0
    value = len(samples) * ORACLE_SAMPLE * args.steps / dt / 1e6
    sample = f"first {ORACLE_SAMPLE} points of each of the two n=2^24 clouds per step (single-threaded C oracle)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": N_POINTS, "sample_points_per_cloud": ORACLE_SAMPLE},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline_leg():
    import oracle

    oracle.build()
    clouds = make_inputs(0)
    s = BASELINE_SAMPLE
    samples = [c[:s].copy() for c in clouds]
    t0 = time.perf_counter()
    for x in samples:
        oracle.hull(x)
    dt = time.perf_counter() - t0
    return {"value": len(samples) * s / dt / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {s} points of each of the two n=2^24 clouds, once (single-threaded C oracle)",
            "seconds": dt, "full_size": full_size_oracle()}


def full_size_oracle():
    """The oracle's own time on the two whole n = 2^24 clouds, as stored with
    its face digests when they were written (one run, single-threaded, on the
    x86 build host, not this machine): the per-point cost grows with n because
    equal-x ties become common, so the 2^19-point sample is faster per point."""
    try:
        with open(os.path.join(ROOT, "tests", "golden", "oracle_hulls.json")) as f:
            g = json.load(f)
        secs = {k: g[k]["oracle_seconds"] for k in ("cube_2e24", "gauss_2e24")}
        return {"seconds": secs, "value": 2 * N_POINTS / sum(secs.values()) / 1e6, "unit": UNIT, "cores": 1,
                "host": "x86 build host (stored with the digests), not the GPU machine"}
    except (OSError, KeyError, ValueError):
        return None


BATCH_CLOUDS = 65536
PLAIN_SAMPLE = 1024  # clouds timed through per-cloud plain launches
ORACLE_BATCH_SAMPLE = 8192  # clouds of the batch hulled by the oracle on all host cores


def face_digest(faces) -> str:
    """SHA-256 of a canonical face list as little-endian int32 rows (a, b, c)."""
    import hashlib

    return hashlib.sha256(np.ascontiguousarray(faces, dtype="<i4").tobytes()).hexdigest()


def _oracle_clouds(chunk):
    """Pool worker: hulls each (cloud index, points) of the chunk with the
    oracle; returns (index, face count, face digest) per cloud."""
    import oracle

    out = []
    for b, x in chunk:
        f = oracle.hull(x)
        out.append((b, int(f.shape[0]), face_digest(f)))
    return out


def batched_cpu_baseline(xyz, off, sample: int = ORACLE_BATCH_SAMPLE, workers: int | None = None,
                         every_cloud: bool = False):
    """The oracle over the first `sample` clouds of the batch, one cloud at a
    time per worker process on every host core (clouds are independent).  The
    pool is started with `spawn` and warmed up (oracle loaded in each worker)
    before the timed map.  With every_cloud, the same pool then hulls the rest
    of the batch, untimed, so that every cloud has a digest.  Returns
    (baseline dict, {cloud: (faces, digest)}); never raises: a failure is
    reported as unavailable with no digests."""
    import multiprocessing as mp

    try:
        import oracle

        oracle.build()
        workers = workers or os.cpu_count() or 1
        sample = min(sample, len(off) - 1)
        clouds = [(b, np.ascontiguousarray(xyz[off[b]: off[b + 1]])) for b in range(sample)]
        per = max(1, len(clouds) // (8 * workers))
        chunks = [clouds[i: i + per] for i in range(0, len(clouds), per)]
        with mp.get_context("spawn").Pool(workers) as pool:
            pool.map_async(_oracle_clouds, [clouds[:1]] * workers, chunksize=1).get(timeout=120)
            t0 = time.perf_counter()
            res = pool.map_async(_oracle_clouds, chunks, chunksize=1).get(timeout=240)
            dt = time.perf_counter() - t0
            if every_cloud and sample < len(off) - 1:
                rest = [(b, np.ascontiguousarray(xyz[off[b]: off[b + 1]])) for b in range(sample, len(off) - 1)]
                res = res + pool.map_async(_oracle_clouds, [rest[i: i + per] for i in range(0, len(rest), per)],
                                           chunksize=1).get(timeout=600)
        digests = {b: (nf, d) for part in res for b, nf, d in part}
        done = min(len(digests), sample)
        return ({"hulls_per_s": done / dt, "cores": workers, "kind": "oracle",
                 "sample": f"first {done} clouds of the batch ({int(off[done] - off[0])} points), one process per core",
                 "seconds": dt}, digests)
    except Exception as e:  # the GPU legs stand without it
        return {"unavailable": f"{type(e).__name__}: {e}"}, {}


def batch_parity(faces, nf, foff, digests) -> dict:
    """Bit-exact check of the batch's per-cloud faces against the oracle's
    digests; raises on the first mismatch."""
    if not digests:
        return {"clouds": 0, "bit_exact": None}
    last = max(digests) + 1
    f = faces[: int(foff[last])].cpu().numpy()
    counts = nf[:last].cpu().numpy()
    for b, (want_nf, want_d) in digests.items():
        got = f[foff[b]: foff[b] + counts[b]]
        if int(counts[b]) != want_nf or face_digest(got) != want_d:
            raise RuntimeError(f"batched faces of cloud {b} differ from the oracle "
                               f"({int(counts[b])} faces, oracle {want_nf})")
    return {"clouds": len(digests), "bit_exact": True}


def batched_leg(hull3d, torch, steps: int, cpu_baseline: bool = False, clouds: int = 0):
    """65,536 independent clouds, sizes round(2^U(4, 12)), distribution drawn
    per cloud: one persistent launch per size class vs per-cloud plain launches.
    clouds > 0 (profiling runs only): that many clouds of the same draw, once."""
    from paper_1205_1171_gb300 import inputs

    xyz, off, kinds = inputs.batch(BATCH_CLOUDS, inputs.seed_for(4))
    if clouds:
        d_xyz = torch.from_numpy(xyz[: off[clouds]]).cuda()
        sizes = np.diff(off[: clouds + 1])
        foff = np.zeros(clouds + 1, np.int64)
        foff[1:] = np.cumsum(np.where(sizes >= 3, 2 * sizes - 4, 0))
        plan = hull3d.Hull3D.tuned(4096, max_clouds=clouds, kind="batch")  # as the batched leg
        faces = torch.empty((int(foff[-1]), 3), dtype=torch.int32, device="cuda")
        nf = torch.zeros(clouds, dtype=torch.int64, device="cuda")
        st = torch.zeros(clouds, dtype=torch.int32, device="cuda")
        plan.batch_async(d_xyz, off[: clouds + 1], faces, foff, nf, st, torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert int((st != 0).sum().item()) == 0
        plan.close()
        return None
    sizes = np.diff(off)
    caps = np.where(sizes >= 3, 2 * sizes - 4, 0)
    foff = np.zeros(len(off), np.int64)
    foff[1:] = np.cumsum(caps)
    d_xyz = torch.from_numpy(xyz).cuda()
    faces = torch.empty((int(foff[-1]), 3), dtype=torch.int32, device="cuda")
    nf = torch.zeros(BATCH_CLOUDS, dtype=torch.int64, device="cuda")
    st = torch.zeros(BATCH_CLOUDS, dtype=torch.int32, device="cuda")
    plan = hull3d.Hull3D.tuned(4096, max_clouds=BATCH_CLOUDS, kind="batch")
    stream = torch.cuda.current_stream()
    plan.batch_async(d_xyz, off, faces, foff, nf, st, stream)
    torch.cuda.synchronize()
    assert int((st != 0).sum().item()) == 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        plan.batch_async(d_xyz, off, faces, foff, nf, st, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    batch_ms = e0.elapsed_time(e1) / steps
    launches = plan.last_launches
    batch_tune = {"knobs": plan.tuned_knobs,
                  "source": "autotuner cache" if plan.tuned_knobs else "library defaults"}
    if plan.tuned_knobs:  # the library defaults on the same batch, for comparison
        dplan = hull3d.Hull3D(4096, max_clouds=BATCH_CLOUDS)
        dplan.batch_async(d_xyz, off, faces, foff, nf, st, stream)
        e0.record(stream)
        for _ in range(steps):
            dplan.batch_async(d_xyz, off, faces, foff, nf, st, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        batch_tune["default_hulls_per_s"] = BATCH_CLOUDS / (e0.elapsed_time(e1) / steps / 1e3)
        dplan.close()
        plan.batch_async(d_xyz, off, faces, foff, nf, st, stream)  # the tuned plan's faces are the ones checked
        torch.cuda.synchronize()
    # per-cloud plain launches on a sample (a rate, so a sample measures it)
    single = hull3d.Hull3D(4096, use_graph=-1)
    pick = np.random.default_rng(0).choice(BATCH_CLOUDS, size=PLAIN_SAMPLE, replace=False)
    views = [(d_xyz[off[b]: off[b + 1]], faces[foff[b]: foff[b + 1]] if caps[b] else faces[:1], nf[b: b + 1],
              st[b: b + 1]) for b in pick]
    for x, f, n1, s1 in views[:16]:
        single.compute_async(x, f, n1, s1, stream)
    torch.cuda.synchronize()
    e0.record(stream)
    for x, f, n1, s1 in views:
        single.compute_async(x, f, n1, s1, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1)
    plan.close()
    single.close()
    total_faces = int(nf.sum().item())
    alg = 12 * len(xyz) + 12 * total_faces  # read every point once, write every face once
    peak, peak_kind = peaks()
    counts = batch_counts(plan.tuned_knobs, BATCH_CLOUDS)
    roof = {"bound": "hbm", "achieved": alg / (batch_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
            "frac": alg / (batch_ms / 1e3) / 1e9 / peak, "traffic": counts and counts["dram_bytes"],
            "peak_kind": peak_kind, "kernel": "k_batch (one cloud per CTA from an atomic queue, four size classes)",
            "alg_bytes_per_batch": alg, "faces": total_faces}
    if counts:
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        ipk = ISSUE_PER_SM_PER_CYCLE * sms * 2070.0 / 1e3
        ach = counts["warp_inst"] / (batch_ms / 1e3) / 1e9
        roof["issue"] = {"bound": "alu", "achieved": ach, "peak": ipk, "unit": "Gwarp-inst/s", "frac": ach / ipk,
                         "active_lanes_per_inst": counts["active_lanes_per_inst"],
                         "peak_basis": f"{ISSUE_PER_SM_PER_CYCLE} warp instructions per SM per cycle x {sms} SMs "
                                       "x 2070 MHz",
                         "counts": "ncu capture of the first 4096 clouds of the same draw, scaled by the clouds"}
    out = {"workload": "65,536 clouds, sizes round(2^U(4,12)) (16..4096), distribution per cloud uniform over "
                       "cube/ball/sphere/gauss", "points": int(len(xyz)), "roofline": roof,
           "hulls_per_s": BATCH_CLOUDS / (batch_ms / 1e3), "ms_per_batch": batch_ms, "launches_per_batch": launches,
           "autotune": batch_tune,
           "per_cloud_plain_hulls_per_s": PLAIN_SAMPLE / (plain_ms / 1e3),
           "per_cloud_plain_sample": PLAIN_SAMPLE}
    if cpu_baseline:
        out["cpu_baseline"], digests = batched_cpu_baseline(xyz, off, every_cloud=True)
        out["parity"] = batch_parity(faces, nf, foff, digests)
    return out


def _cloud_mismatch(fa, na, fb, nb, foff):
    """Per cloud: True where the two face lists (rows foff[b] ..) differ."""
    rows = np.zeros(len(fa), bool)
    rows[:] = (fa != fb).any(axis=1)
    B = len(na)
    wrong = na != nb
    for b in np.flatnonzero(~wrong):
        k = int(na[b])
        if k and rows[foff[b]: foff[b] + k].any():
            wrong[b] = True
    return wrong


def float32_ablation_leg(hull3d, torch):
    """The paper's float32 arithmetic (Sec. 3, cl_float coordinates) against
    the exact predicates, on the batch kernel: the fraction of clouds whose
    faces differ from the exact faces (themselves checked against the oracle
    in the tests and the batched leg), or that fail, on the 65,536-cloud batch
    and on 1,024 seeded 4096-point cubes."""
    from paper_1205_1171_gb300 import inputs

    out = {"arith": "float32 coordinates, cross products, quotient times and comparisons (no perturbation)",
           "kernel": "k_batch (clouds of at most 4096 points)"}
    cases = {"batch_65536": inputs.batch(BATCH_CLOUDS, inputs.seed_for(4))}
    cubes = [inputs.cloud_seeded("cube", 4096, inputs.seed_for(1) + 7919 * i) for i in range(1024)]
    off = np.arange(0, 4096 * 1025, 4096, dtype=np.int64)
    cases["cube4096_x1024"] = (np.concatenate(cubes), off, ["cube"] * 1024)
    for name, (xyz, off, kinds) in cases.items():
        B = len(off) - 1
        sizes = np.diff(off)
        foff = np.zeros(B + 1, np.int64)
        foff[1:] = np.cumsum(np.where(sizes >= 3, 2 * sizes - 4, 0))
        d_xyz = torch.from_numpy(xyz).cuda()
        res = []
        for f32 in (0, 1):
            plan = hull3d.Hull3D(4096, max_clouds=B, float32_ablation=f32)
            faces = torch.full((int(foff[-1]), 3), -1, dtype=torch.int32, device="cuda")
            nf = torch.zeros(B, dtype=torch.int64, device="cuda")
            st = torch.zeros(B, dtype=torch.int32, device="cuda")
            plan.batch_async(d_xyz, off, faces, foff, nf, st)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            plan.batch_async(d_xyz, off, faces, foff, nf, st)
            e1.record()
            torch.cuda.synchronize()
            res.append((faces.cpu().numpy(), nf.cpu().numpy(), st.cpu().numpy(), e0.elapsed_time(e1)))
            plan.close()
        (fe, ne, se, me), (ff, nff, sf, mf) = res
        assert not se.any(), "exact batch failed"
        failed = sf != 0
        wrong = _cloud_mismatch(fe, ne, ff, nff, foff) & ~failed
        rec = {"clouds": B, "wrong": int(wrong.sum()), "failed": int(failed.sum()),
               "wrong_or_failed_frac": float((wrong | failed).mean()),
               "exact_hulls_per_s": B / (me / 1e3), "float32_hulls_per_s": B / (mf / 1e3)}
        kinds = np.array(kinds)
        rec["by_dist"] = {d: float((wrong | failed)[kinds == d].mean()) for d in sorted(set(kinds.tolist()))}
        cls = np.digitize(sizes, [257, 1025, 2049])
        rec["by_size_class"] = {lab: float((wrong | failed)[cls == c].mean()) for c, lab in
                                enumerate(("16-256", "257-1024", "1025-2048", "2049-4096")) if (cls == c).any()}
        out[name] = rec
    return out


def _time_ms(torch, fn, reps: int, stream) -> float:
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def adjacency_leg(hull3d, torch, plan, faces, nfs, n_points, stream, reps: int = 5):
    """Face neighbours and vertex stars (hull3d_adjacency_async) of the main
    leg's hulls and of a 2^20-point sphere's (about 2.1 million faces)."""
    from paper_1205_1171_gb300 import inputs

    peak, peak_kind = peaks()
    out = {}

    def one(p, f, nf, n, label):
        F = f.shape[0]
        nb = torch.empty((F, 3), dtype=torch.int32, device="cuda")
        off = torch.empty(n + 1, dtype=torch.int64, device="cuda")
        star = torch.empty(3 * F, dtype=torch.int32, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        ms = _time_ms(torch, lambda: p.adjacency_async(f, nf, n, nb, off, star, st, stream), reps, stream)
        assert int(st.item()) == 0, "adjacency status"
        faces_n = int(nf.item())
        alg = 12 * faces_n + 12 * faces_n + 8 * (n + 1) + 12 * faces_n  # faces in; neighbours, offsets, stars out
        out[label] = {"faces": faces_n, "ms": ms, "alg_bytes": alg, "gbs": alg / (ms / 1e3) / 1e9,
                      "frac_of_hbm": alg / (ms / 1e3) / 1e9 / peak, "launches": p.last_launches}

    for k, (f, nf) in enumerate(zip(faces, nfs)):
        one(plan, f, nf, n_points, f"hull_2e24_{k}")
    sph = torch.from_numpy(inputs.cloud_seeded("sphere", 1 << 20, inputs.seed_for(2))).cuda()
    sp = hull3d.Hull3D(1 << 20)
    fs = sp.compute(sph)
    one(sp, fs, torch.tensor([fs.shape[0]], dtype=torch.int64, device="cuda"), 1 << 20, "sphere_2e20")
    sp.close()
    out["peak"] = peak
    out["peak_kind"] = peak_kind
    return out


def delaunay_leg(hull3d, torch, stream):
    """2D Delaunay triangulation through the lifting map (hull3d_delaunay_async)
    of 2^20 and 2^22 points uniform in a disk."""
    from paper_1205_1171_gb300 import inputs

    out = {"input": "points uniform in the disk of radius 2^15 - 1 (int32), seed_for(60)"}
    for n in (1 << 20, 1 << 22):
        pts = torch.from_numpy(inputs.planar_seeded("disk", n, inputs.seed_for(60))).cuda()
        p = hull3d.Hull3D(n)
        tris = torch.empty((2 * n, 3), dtype=torch.int32, device="cuda")
        nt = torch.zeros(1, dtype=torch.int64, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        ms = _time_ms(torch, lambda: p.delaunay_async(pts, tris, nt, st, stream), 3, stream)
        assert int(st.item()) == 0, "delaunay status"
        out[f"n_{n}"] = {"ms": ms, "mpoints_per_s": n / ms / 1e3, "triangles": int(nt.item()),
                         "launches": p.last_launches}
        p.close()
    return out


SERVE_RATE = 20000.0     # requests per second (Poisson)
SERVE_REQUESTS = 4000    # arrivals measured, the same ones for both forms


def serving_leg(hull3d, torch):
    """Open-loop Poisson stream of hull requests, sizes round(2^U(6, 18)), mixed
    distributions, 8 GB budget: continuous batching vs one request at a time,
    both fed the same first SERVE_REQUESTS arrivals of the stream."""
    from paper_1205_1171_gb300 import serve

    pool = serve.request_pool(256, inputs_seed(5))
    arrivals = serve.poisson_arrivals(SERVE_RATE, 2.0 * SERVE_REQUESTS / SERVE_RATE, np.random.default_rng(6))
    arrivals = arrivals[:SERVE_REQUESTS]
    picks = np.random.default_rng(7).integers(0, len(pool), size=len(arrivals))
    with serve.HullServer(budget_bytes=8 << 30) as srv:
        warm = [srv.submit(c) for c in pool[:32]]
        for f in warm:
            f.result()
        srv.stats = serve.Stats()
        futs = serve.replay(srv.submit, arrivals, pool, picks)
        for f in futs:
            f.result()
        served = srv.stats.summary()
        srv_knobs = srv.backend.knobs
    plan = hull3d.Hull3D(1 << 18)
    lat = []
    host = [torch.from_numpy(pool[k]).pin_memory() for k in range(len(pool))]
    out = torch.empty((1 << 19, 3), dtype=torch.int32).pin_memory()
    for k in range(8):
        plan.compute_host(host[k], out)
    t0 = time.perf_counter()
    for t, k in zip(arrivals, picks):
        while time.perf_counter() < t0 + t:
            pass
        plan.compute_host(host[k], out)
        lat.append(time.perf_counter() - (t0 + t))
    span = time.perf_counter() - t0
    plan.close()
    lat = np.array(lat) * 1e3
    pts = float(np.mean([len(pool[k]) for k in picks]))
    window = float(arrivals[-1])
    return {"workload": f"Poisson {SERVE_RATE:.0f} req/s, sizes round(2^U(6,18)), mixed distributions, 8 GB budget, "
                        "requests drawn from 256 distinct clouds",
            "requests": int(len(arrivals)), "arrival_window_s": window,
            "shortened": f"the first {len(arrivals)} arrivals ({window:.2f} s of the stream) instead of 10 s: the "
                         "offered load is above what one GPU hulls, so a longer window only lengthens the backlog "
                         "(and the one-at-a-time replay of 200k requests would take minutes); both forms get the "
                         "same arrivals",
            "served": served, "served_knobs": srv_knobs,
            "one_at_a_time": {"requests": int(len(lat)), "p50_ms": float(np.percentile(lat, 50)),
                              "p99_ms": float(np.percentile(lat, 99)), "hulls_per_s": len(lat) / span},
            "mean_points_per_request": pts}


def inputs_seed(k: int) -> int:
    from paper_1205_1171_gb300 import inputs

    return inputs.seed_for(k)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fused", type=int, default=0, help="fused bottom levels (0 = library default)")
    ap.add_argument("--occ", type=int, default=0, help="global merge kernel occupancy knob (1 or 4)")
    ap.add_argument("--cmp-level", type=int, default=0, help="first level of the compacted warp kernel (0 = default)")
    ap.add_argument("--n", type=int, default=1 << 24, help="points per cloud (profiling runs only; default 2^24)")
    ap.add_argument("--dists", default=",".join(DISTS), help="clouds per step (profiling runs only)")
    ap.add_argument("--seg-level", type=int, default=0, help="first time-segment-parallel level (0 = default)")
    ap.add_argument("--seg-events", type=int, default=0, help="child events per time window (0 = default)")
    ap.add_argument("--no-batched", action="store_true", help="skip the 65,536-cloud batched measurement")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving measurement")
    ap.add_argument("--no-ablation", action="store_true", help="skip the float32 arithmetic ablation")
    ap.add_argument("--no-extras", action="store_true", help="skip the adjacency and Delaunay timings")
    ap.add_argument("--profile-once", action="store_true",
                    help="profiling runs only: hull each cloud once (no warm-up, no timing) and exit")
    ap.add_argument("--batch-only", type=int, default=0,
                    help="profiling runs only: run the batched leg on this many clouds once and exit")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    npts = args.n

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch

    from paper_1205_1171_gb300 import build, hull3d

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    if args.batch_only:
        batched_leg(hull3d, torch, 1, clouds=args.batch_only)
        return
    dists = tuple(args.dists.split(","))
    clouds = make_inputs(rank, npts, dists)
    dev_clouds = [torch.from_numpy(c).cuda() for c in clouds]
    cli_knobs = dict(fused_levels=args.fused, level_occupancy=args.occ, cmp_level=args.cmp_level,
                     seg_level=args.seg_level, seg_events=args.seg_events)
    default_plan = not any(cli_knobs.values())
    # the plan a user gets from Hull3D.tuned (the autotuner's knobs for this
    # GPU, size and distribution class; the library defaults where none)
    plan = hull3d.Hull3D.tuned(npts, dist_class="volume") if default_plan else hull3d.Hull3D(npts, **cli_knobs)
    tuned_knobs = getattr(plan, "tuned_knobs", {}) if default_plan else {}
    plan_knobs = dict(tuned_knobs) if default_plan else {k: v for k, v in cli_knobs.items() if v}
    cap = 2 * npts - 4
    faces = [torch.empty((cap, 3), dtype=torch.int32, device="cuda") for _ in clouds]
    nfs = [torch.zeros(1, dtype=torch.int64, device="cuda") for _ in clouds]
    sts = [torch.zeros(1, dtype=torch.int32, device="cuda") for _ in clouds]
    stream = torch.cuda.current_stream()
    if args.profile_once:
        for x, f, nf, st in zip(dev_clouds, faces, nfs, sts):
            plan.compute_async(x, f, nf, st, stream)
        torch.cuda.synchronize()
        assert all(int(st.item()) == 0 for st in sts), "device status"
        plan.close()
        return

    def step():
        launches = 0
        for x, f, nf, st in zip(dev_clouds, faces, nfs, sts):
            plan.compute_async(x, f, nf, st, stream)
            launches += plan.last_launches
        return launches

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    for st in sts:
        assert int(st.item()) == 0, "device status"
    nface = [int(nf.item()) for nf in nfs]
    level_ev = []
    for x in dev_clouds:  # per-level movie lengths of each cloud (statistics for the roofline)
        plan.compute_async(x, faces[0], nfs[0], sts[0], stream)
        level_ev.append(plan.level_events())

    # the timed region replays the plan's cached CUDA graphs (the path a user's
    # hull3d_compute_async takes); nothing is recorded inside it
    clocks = ClockSampler(torch.cuda.current_device())
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    launches = 0
    for _ in range(args.steps):
        launches += step()
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    clk = clocks.stop()
    # per-phase and per-level times: a separate profiled pass over the same
    # clouds right after it (plain launches with CUDA events recorded on the
    # launching stream at every phase and level boundary)
    plan.profile(True)
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(args.steps):
        step()
    p1.record(stream)
    torch.cuda.synchronize()
    profiled_ms = p0.elapsed_time(p1)
    level_ms = plan.profile_levels()
    phase_ms, calls = plan.profile_read()
    plan.profile(False)
    ms = max_over_ranks(ms, dist)
    if dist:
        dist.barrier()
    points = len(clouds) * npts * args.steps * world
    value = points / (ms / 1e3) / 1e6

    # end to end through the public API from pinned host memory
    host_in = [torch.from_numpy(c).pin_memory() for c in clouds]
    host_out = torch.empty((cap, 3), dtype=torch.int32).pin_memory()
    for x in host_in:
        plan.compute_host(x, host_out)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    d2h = 0
    for _ in range(args.steps):
        for x in host_in:
            f = plan.compute_host(x, host_out)
            d2h += f.shape[0] * 12 + 12
    e_dt = time.perf_counter() - e0
    e_dt = max_over_ranks(e_dt, dist)
    e2e = {"value": points / e_dt / 1e6, "unit": UNIT, "h2d_bytes_per_step": 12 * npts * len(clouds),
           "d2h_bytes_per_step": d2h // args.steps}

    # roofline of the dominant kernel -- the thread-per-merge level kernel, which
    # runs the levels below the compacted ones -- from the per-level events
    # recorded live on the launching stream in the timed region
    peak, peak_kind = peaks()
    o = plan.opts
    steps = max(args.steps, 1)
    L = int(np.ceil(np.log2(npts)))
    # k_level runs from level 3 (level 2 has its own kernel) below the compacted levels
    klev = [lv for lv in range(max(3, plan.fused_levels_used + 1), L + 1) if lv < o["cmp_level"]]
    k_bytes = sum(level_alg_bytes(npts, ev, lv) for ev in level_ev for lv in klev)  # per step
    k_ms = sum(float(level_ms[lv]) for lv in klev) / steps
    k_launches = len(klev) * len(clouds)
    achieved = k_bytes / (k_ms / 1e3) / 1e9 if k_ms > 0 else 0.0
    ab = [alg_bytes(npts, ev, plan.fused_levels_used, nf, o["seg_level"]) for ev, nf in zip(level_ev, nface)]
    alg = {k: sum(a[k] for a in ab) for k in ab[0]}  # bytes per step
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": kernel_traffic(npts, dists, plan_knobs),
                "kernel": "k_level (one thread per merge)",
                "levels": [klev[0], klev[-1]] if klev else [], "launches_per_step": k_launches,
                "alg_bytes_per_launch": k_bytes / max(k_launches, 1), "ms_per_launch": k_ms / max(k_launches, 1),
                "peak_kind": peak_kind,
                "timing": "kernel and phase times from a profiled pass over the same clouds right after the timed "
                          "region (plain launches, CUDA events at each level boundary on the launching stream); "
                          "the timed region replays CUDA graphs",
                "profiled_pass_ms_per_step": profiled_ms / steps,
                "phase_ms_per_step": {k: v / steps for k, v in phase_ms.items()},
                "phase_alg_bytes_per_step": alg,
                "phase_gbs": {k: alg[k] / (phase_ms[k] / steps / 1e3) / 1e9 for k in alg if phase_ms[k] > 0}}
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    sm_mhz = (clk or {}).get("sm_mhz") or (clk or {}).get("sm_max_mhz") or 2070.0
    roofline["issue"] = kernel_issue(k_ms / max(k_launches, 1), sms, float(sm_mhz), npts, dists, plan_knobs)
    autotune_rec = {"knobs": tuned_knobs, "source": "autotuner cache" if tuned_knobs else "library defaults"}
    if tuned_knobs:  # the same steps on a plan with the library defaults, for comparison
        dplan = hull3d.Hull3D(npts)
        for _ in range(2):
            for x, f, nf, st in zip(dev_clouds, faces, nfs, sts):
                dplan.compute_async(x, f, nf, st, stream)
        torch.cuda.synchronize()
        d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        d0.record(stream)
        for _ in range(args.steps):
            for x, f, nf, st in zip(dev_clouds, faces, nfs, sts):
                dplan.compute_async(x, f, nf, st, stream)
        d1.record(stream)
        torch.cuda.synchronize()
        autotune_rec["default_value"] = len(clouds) * npts * args.steps / (d0.elapsed_time(d1) / 1e3) / 1e6
        dplan.close()

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": npts, "clouds_per_step": len(clouds),
                       "faces": nface, "l2": "inputs larger than L2 (201 MB per cloud), no flush",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "clocks": clk, "e2e": e2e, "gpu_launches": launches, "roofline": roofline, "autotune": autotune_rec}
    if not args.no_extras and rank == 0:
        line["adjacency"] = adjacency_leg(hull3d, torch, plan, faces, nfs, npts, stream)
        line["delaunay"] = delaunay_leg(hull3d, torch, stream)
    if not args.no_batched:
        b = batched_leg(hull3d, torch, max(1, args.steps // 2),
                        cpu_baseline=rank == 0 and world == 1 and not args.no_cpu_baseline)
        if dist:
            b["hulls_per_s"] = world * BATCH_CLOUDS / (max_over_ranks(b["ms_per_batch"], dist) / 1e3)
        line["batched"] = b
    if not args.no_serving and rank == 0:
        line["serving"] = serving_leg(hull3d, torch)
    if not args.no_ablation and rank == 0:
        line["float32_ablation"] = float32_ablation_leg(hull3d, torch)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_leg()
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
