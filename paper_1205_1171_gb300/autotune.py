"""Autotuner for the speed knobs of the hull pipeline.

None of the knobs changes the result (the faces are the perturbed hull's,
whatever the schedule); they only choose which kernel merges which level:
  cmp_level        first level merged one warp per merge (compacted tables)
  seg_level        first level whose large merges are split into time windows
  seg_events       child events per time window (the segment length)
  seg_min_events   merges with fewer child events skip the windows
  level_occupancy  register cap of the thread-per-merge kernel (1 or 4)
The tuner times each candidate on seeded synthetic clouds of every
distribution for an n-bucket (n rounded up to a power of two), keeps the one
with the lowest total time, and stores it in a JSON cache keyed by GPU name
and bucket.  Hull3D.tuned(n) then plans with the cached knobs.
"""
from __future__ import annotations

import itertools
import json
import math
import os
import time
from typing import Callable, Iterable

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "tuning.json")
KNOBS = ("cmp_level", "seg_level", "seg_events", "seg_min_events", "level_occupancy")


def bucket(n: int) -> int:
    """log2 of n rounded up (the cache is keyed by it)."""
    return max(1, int(math.ceil(math.log2(max(n, 2)))))


def candidates(n: int) -> list[dict]:
    """The search space for hulls of about n points (levels above log2 n do nothing).
    0 keeps the library's automatic choice: for cmp_level the size rule, for
    seg_min_events the per-level rule, for level_occupancy the per-level caps."""
    L = bucket(n)
    cmp_levels = sorted({0} | {min(L + 1, c) for c in (max(6, L - 12), max(6, L - 10), 13)})
    seg_levels = sorted({min(L + 1, s) for s in (8, 10, 12, 64)})
    out = []
    for cl, sl, K, smin, occ in itertools.product(cmp_levels, seg_levels, (256, 512, 1024), (0, 256, 512), (0, 4)):
        if sl > L and (K != 512 or smin != 0):
            continue  # windows never used: one representative
        out.append(dict(cmp_level=cl, seg_level=sl, seg_events=K, seg_min_events=smin, level_occupancy=occ))
    return out


def key(gpu_name: str, n: int) -> str:
    return f"{gpu_name}|2^{bucket(n)}"


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


def lookup(gpu_name: str, n: int, path: str = DEFAULT_CACHE) -> dict | None:
    """Tuned knobs for the bucket of n, or for the nearest tuned bucket below."""
    cache = load(path)
    b = bucket(n)
    for bb in range(b, 0, -1):
        e = cache.get(f"{gpu_name}|2^{bb}")
        if e:
            return {k: e["knobs"][k] for k in KNOBS if k in e["knobs"]}
    return None


def search(space: Iterable[dict], measure: Callable[[dict], float]) -> tuple[dict, float, list]:
    """Times every candidate with measure(knobs) -> ms; returns (best, ms, all)."""
    results = []
    for kn in space:
        ms = measure(kn)
        results.append((ms, kn))
    results.sort(key=lambda r: r[0])
    return results[0][1], results[0][0], results


def tune(n: int, reps: int = 2, dists: Iterable[str] | None = None, space: Iterable[dict] | None = None,
         path: str = DEFAULT_CACHE, max_candidates: int | None = None, verbose: bool = False) -> dict:
    """Tunes the bucket of n on the current CUDA device and updates the cache."""
    import torch

    from paper_1205_1171_gb300 import hull3d, inputs

    dists = tuple(dists or inputs.DISTS)
    N = 1 << bucket(n)
    clouds = [torch.from_numpy(inputs.cloud_seeded(d, N, inputs.seed_for(40 + i))).cuda() for i, d in enumerate(dists)]
    faces = torch.empty((2 * N, 3), dtype=torch.int32, device="cuda")
    nf = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    space = list(space or candidates(N))
    if max_candidates:
        space = space[:max_candidates]

    def measure(kn: dict) -> float:
        p = hull3d.Hull3D(N, **kn)
        try:
            for x in clouds:  # warm up (captures the graphs)
                p.compute_async(x, faces, nf, st)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
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
    name = torch.cuda.get_device_name()
    cache = load(path)
    cache[key(name, N)] = {"knobs": best, "ms_per_step": ms, "dists": list(dists), "n": N,
                           "candidates": len(allr), "tuned_s": round(time.time() - t0, 1)}
    save(cache, path)
    return best


def main():
    import argparse

    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--n", type=int, action="append", required=True, help="hull size (repeatable)")
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--out", default=DEFAULT_CACHE)
    ap.add_argument("--max-candidates", type=int, default=None)
    a = ap.parse_args()
    for n in a.n:
        print(json.dumps({"n": n, "best": tune(n, a.reps, path=a.out, max_candidates=a.max_candidates,
                                               verbose=True)}), flush=True)


if __name__ == "__main__":
    main()
