"""Autotuner for the speed knobs of the hull pipeline.

None of the knobs changes the result (the faces are the perturbed hull's,
whatever the schedule); they only choose which kernel merges which level and
how work is grouped:
  single hulls and groups of large clouds (kind "single", "multi"):
    cmp_level        first level merged one warp per merge (compacted tables)
    seg_level        first level whose large merges are split into time windows
    seg_events       child events per time window (the segment length)
    seg_min_events   merges with fewer child events skip the windows
    level_occupancy  register cap of the thread-per-merge kernel (1 or 4)
  groups of large clouds also (kind "multi"):
    multi_ranks      rank space of one group (how many clouds share its launches)
  batches of small clouds (kind "batch"):
    batch_warp_nodes the batch kernel's cut-over from one thread per merge to
                     one warp per merge (merges of a level of a cloud)
The tuner times each candidate on seeded synthetic clouds of one distribution
class for an n-bucket (n rounded up to a power of two): "volume" (cube, ball,
clipped Gaussian: few points on the hull) or "surface" (points on a sphere:
nearly all on the hull), keeps the one with the lowest time, and stores it in
a JSON cache keyed by GPU name, kind, bucket and class.  Hull3D.tuned() then
plans with the cached knobs.  A cache measured on this library's target GPU
ships with the package (tuning_gb300.json); a local cache (written by tune())
takes precedence.
"""
from __future__ import annotations

import itertools
import json
import math
import os
import time
from typing import Callable, Iterable

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_CACHE = os.path.join(HERE, "_build", "tuning.json")
SHIPPED_CACHE = os.path.join(HERE, "tuning_gb300.json")
KNOBS = ("cmp_level", "seg_level", "seg_events", "seg_min_events", "level_occupancy", "seg_events_min")
KIND_KNOBS = {"single": KNOBS, "multi": KNOBS + ("multi_ranks",), "batch": ("batch_warp_nodes",)}
CLASSES = {"volume": ("cube", "ball", "gauss"), "surface": ("sphere",)}


def dist_class(dist: str) -> str:
    """The distribution class of a named distribution."""
    return "surface" if dist == "sphere" else "volume"


def bucket(n: int) -> int:
    """log2 of n rounded up (the cache is keyed by it)."""
    return max(1, int(math.ceil(math.log2(max(n, 2)))))


def candidates(n: int) -> list[dict]:
    """The search space for hulls of about n points (levels above log2 n do nothing).
    0 keeps the library's automatic choice: for cmp_level the size rule, for
    seg_min_events the per-level rule, for level_occupancy the per-level caps."""
    L = bucket(n)
    cmp_levels = sorted({0} | {min(L + 1, c) for c in (max(6, L - 12), max(6, L - 10), 13)}
                        | ({3, 4} if L <= 16 else set()))  # small hulls: the warp kernel from low levels
    seg_levels = sorted({min(L + 1, s) for s in (8, 10, 12, 64)})
    out = [dict(cmp_level=0, seg_level=0, seg_events=0, seg_min_events=0, level_occupancy=0, seg_events_min=0)]
    for cl, sl, K, smin, occ, kmin in itertools.product(cmp_levels, seg_levels, (256, 512, 1024), (0, 256, 512),
                                                        (0, 4), (0, 32)):
        if sl > L and (K != 512 or smin != 0 or kmin != 0):
            continue  # windows never used: one representative
        out.append(dict(cmp_level=cl, seg_level=sl, seg_events=K, seg_min_events=smin, level_occupancy=occ,
                        seg_events_min=kmin))
    return out


def key(gpu_name: str, n: int, cls: str | None = None, kind: str = "single") -> str:
    k = f"{gpu_name}|2^{bucket(n)}"
    if cls:
        k += f"|{cls}"
    if kind != "single":
        k += f"|{kind}"
    return k


def load(path: str = DEFAULT_CACHE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save(cache: dict, path: str = DEFAULT_CACHE) -> None:
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def lookup(gpu_name: str, n: int, path: str | None = DEFAULT_CACHE, cls: str | None = None, kind: str = "single",
           shipped: str | None = None) -> dict | None:
    """Tuned knobs of a kind for the bucket of n and the class (else any
    class), or for the nearest tuned bucket below; the cache at `path` first,
    then the shipped one (shipped=None: the package's)."""
    names = KIND_KNOBS[kind]
    for src in (path, shipped if shipped is not None else SHIPPED_CACHE):
        if not src:
            continue
        cache = load(src)
        for bb in range(bucket(n), 0, -1):
            for c in ([cls] if cls else []) + [None]:
                e = cache.get(key(gpu_name, 1 << bb, c, kind))
                if e:
                    return {k: e["knobs"][k] for k in names if k in e["knobs"]}
    return None


def search(space: Iterable[dict], measure: Callable[..., float]) -> tuple[dict, float, list]:
    """Times every candidate with measure(knobs, limit) -> ms, where limit is
    a time (ms) past which the candidate may stop early (it cannot be the
    best); returns (best, ms, all)."""
    import inspect

    takes_limit = len(inspect.signature(measure).parameters) > 1
    results = []
    best = float("inf")
    for kn in space:
        ms = measure(kn, 4.0 * best) if takes_limit else measure(kn)
        best = min(best, ms)
        results.append((ms, kn))
    results.sort(key=lambda r: r[0])
    return results[0][1], results[0][0], results


def _store(path: str, k: str, entry: dict) -> None:
    cache = load(path)
    cache[k] = entry
    save(cache, path)


def tune(n: int, reps: int = 2, dists: Iterable[str] | None = None, space: Iterable[dict] | None = None,
         path: str = DEFAULT_CACHE, max_candidates: int | None = None, verbose: bool = False,
         cls: str | None = None) -> dict:
    """Tunes single hulls of the bucket of n (and class cls) on the current
    CUDA device and updates the cache."""
    import torch

    from paper_1205_1171_gb300 import hull3d, inputs

    dists = tuple(dists or (CLASSES[cls] if cls else inputs.DISTS))
    N = 1 << bucket(n)
    clouds = [torch.from_numpy(inputs.cloud_seeded(d, N, inputs.seed_for(40 + i))).cuda() for i, d in enumerate(dists)]
    faces = torch.empty((2 * N, 3), dtype=torch.int32, device="cuda")
    nf = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    space = list(space or candidates(N))
    if max_candidates:
        space = space[:max_candidates]

    def measure(kn: dict, limit: float = float("inf")) -> float:
        p = hull3d.Hull3D(N, **kn)
        try:
            for x in clouds:  # warm up (captures the graphs)
                p.compute_async(x, faces, nf, st)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for x in clouds:
                p.compute_async(x, faces, nf, st)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            if ms <= limit:  # a slow candidate is not repeated
                e0.record()
                for _ in range(reps):
                    for x in clouds:
                        p.compute_async(x, faces, nf, st)
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / reps
        finally:
            p.close()
        if verbose:
            print(f"{ms:9.2f} ms  {kn}", flush=True)
        return ms

    t0 = time.time()
    best, ms, allr = search(space, measure)
    _store(path, key(torch.cuda.get_device_name(), N, cls), {
        "knobs": best, "ms_per_step": ms, "dists": list(dists), "n": N, "candidates": len(allr),
        "default_ms": next((m for m, kn in allr if all(v == 0 for v in kn.values())), None),
        "tuned_s": round(time.time() - t0, 1)})
    return best


def batch_candidates() -> list[dict]:
    return [dict(batch_warp_nodes=w) for w in (8, 16, 32, 64, 128, 256, 1 << 20)]


def tune_batch(clouds: int = 8192, reps: int = 3, path: str = DEFAULT_CACHE, verbose: bool = False,
               space: Iterable[dict] | None = None) -> dict:
    """Tunes the batch kernel's cut-over on the first `clouds` clouds of the
    seeded batch draw (sizes round(2^U(4, 12)), mixed distributions)."""
    import numpy as np
    import torch

    from paper_1205_1171_gb300 import hull3d, inputs

    xyz, off, _ = inputs.batch(clouds, inputs.seed_for(44))
    sizes = np.diff(off)
    foff = np.zeros(len(off), np.int64)
    foff[1:] = np.cumsum(np.where(sizes >= 3, 2 * sizes - 4, 0))
    d_xyz = torch.from_numpy(xyz).cuda()
    faces = torch.empty((max(int(foff[-1]), 1), 3), dtype=torch.int32, device="cuda")
    nf = torch.zeros(clouds, dtype=torch.int64, device="cuda")
    st = torch.zeros(clouds, dtype=torch.int32, device="cuda")

    def measure(kn: dict) -> float:
        p = hull3d.Hull3D(4096, max_clouds=clouds, **kn)
        try:
            p.batch_async(d_xyz, off, faces, foff, nf, st)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                p.batch_async(d_xyz, off, faces, foff, nf, st)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
        finally:
            p.close()
        if verbose:
            print(f"{ms:9.2f} ms  {kn}", flush=True)
        return ms

    t0 = time.time()
    best, ms, allr = search(list(space or batch_candidates()), measure)
    _store(path, key(torch.cuda.get_device_name(), 4096, None, "batch"), {
        "knobs": best, "ms_per_batch": ms, "clouds": clouds, "candidates": len(allr),
        "default_ms": next((m for m, kn in allr if kn.get("batch_warp_nodes") == 64), None),
        "tuned_s": round(time.time() - t0, 1)})
    return best


def multi_candidates(ranks: int) -> list[dict]:
    L = bucket(ranks)
    out = []
    for cl, sl, mr in itertools.product((0, max(6, L - 12), 9, 13), (8, 10, 12), (0, ranks // 2, ranks // 4)):
        out.append(dict(cmp_level=cl, seg_level=sl, seg_events=0, seg_min_events=0, level_occupancy=0,
                        multi_ranks=mr))
    return out


def tune_multi(ranks: int = 1 << 21, clouds: int = 128, reps: int = 2, path: str = DEFAULT_CACHE,
               verbose: bool = False, space: Iterable[dict] | None = None) -> dict:
    """Tunes groups of large clouds (sizes round(2^U(12.01, 18)), mixed
    distributions, as a server's large requests) for a plan of `ranks` ranks."""
    import numpy as np
    import torch

    from paper_1205_1171_gb300 import hull3d, inputs

    rng = np.random.default_rng(inputs.seed_for(45))
    sizes = np.round(2.0 ** rng.uniform(12.01, 18.0, clouds)).astype(np.int64)
    kinds = rng.integers(0, len(inputs.DISTS), clouds)
    pts = [inputs.cloud_seeded(inputs.DISTS[k], int(n), inputs.seed_for(46) + i) for i, (n, k) in
           enumerate(zip(sizes, kinds))]
    off = np.zeros(clouds + 1, np.int64)
    off[1:] = np.cumsum(sizes)
    foff = np.zeros(clouds + 1, np.int64)
    foff[1:] = np.cumsum(2 * sizes - 4)
    d_xyz = torch.from_numpy(np.concatenate(pts)).cuda()
    faces = torch.empty((int(foff[-1]), 3), dtype=torch.int32, device="cuda")
    nf = torch.zeros(clouds, dtype=torch.int64, device="cuda")
    st = torch.zeros(clouds, dtype=torch.int32, device="cuda")

    def measure(kn: dict) -> float:
        p = hull3d.Hull3D(ranks, max_clouds=clouds, **kn)
        try:
            p.batch_async(d_xyz, off, faces, foff, nf, st)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                p.batch_async(d_xyz, off, faces, foff, nf, st)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
        finally:
            p.close()
        if verbose:
            print(f"{ms:9.2f} ms  {kn}", flush=True)
        return ms

    t0 = time.time()
    best, ms, allr = search(list(space or multi_candidates(ranks)), measure)
    _store(path, key(torch.cuda.get_device_name(), ranks, None, "multi"), {
        "knobs": best, "ms_per_batch": ms, "clouds": clouds, "ranks": ranks, "candidates": len(allr),
        "default_ms": next((m for m, kn in allr if all(v == 0 for v in kn.values())), None),
        "tuned_s": round(time.time() - t0, 1)})
    return best


def main():
    import argparse

    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--n", type=int, action="append", default=[], help="single-hull size (repeatable)")
    ap.add_argument("--cls", choices=sorted(CLASSES), default=None, help="distribution class of --n")
    ap.add_argument("--batch", type=int, default=0, help="tune the batch kernel on this many clouds")
    ap.add_argument("--multi", type=int, default=0, help="tune groups of large clouds for this rank space")
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--out", default=DEFAULT_CACHE)
    ap.add_argument("--max-candidates", type=int, default=None)
    a = ap.parse_args()
    for n in a.n:
        print(json.dumps({"n": n, "cls": a.cls, "best": tune(n, a.reps, path=a.out, max_candidates=a.max_candidates,
                                                              verbose=True, cls=a.cls)}), flush=True)
    if a.batch:
        print(json.dumps({"batch": a.batch, "best": tune_batch(a.batch, path=a.out, verbose=True)}), flush=True)
    if a.multi:
        print(json.dumps({"multi": a.multi, "best": tune_multi(a.multi, path=a.out, verbose=True)}), flush=True)


if __name__ == "__main__":
    main()
