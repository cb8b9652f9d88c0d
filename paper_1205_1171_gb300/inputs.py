"""Seeded synthetic point clouds shaped like the paper's workloads.

The paper (Sec. 4) times n = 4 ... 2^23 points but never states their
distribution, so these generators stand in for it.  They hold none of the hull
arithmetic and are the only module shared by the CUDA path's tests, the
benchmark and the CPU oracle's tests.

Every cloud is int32 with coordinates in [-2^20, 2^20) and no duplicate
points (duplicates are redrawn).  Distributions:

* ``cube``   uniform integers in the cube [-2^20, 2^20)^3;
* ``ball``   cube samples kept when x^2 + y^2 + z^2 < 2^40;
* ``sphere`` standard normal 3-vectors, normalised, scaled by 2^20 - 1 and
  rounded (almost every point on the hull);
* ``gauss``  rint(N(0, (2^18)^2)) per coordinate, clipped to the cube (a few
  hundred points land on each clipping plane: coplanar hull facets).

Planar point sets for the Delaunay triangulation (``planar_seeded``), int32
(x, y) with |x|, |y| < 2^15, no duplicates:

* ``square`` uniform integers in [-2^15 + 1, 2^15 - 1]^2;
* ``disk``   square samples kept inside the radius 2^15 - 1;
* ``gauss``  rint(N(0, (2^13)^2)) per coordinate, clipped to the square (points
  on the clipping edges: collinear boundary runs);
* ``grid``   distinct points of a jittered-free integer lattice with a random
  origin and spacing (every four neighbours cocircular).
"""
from __future__ import annotations

import numpy as np

LO = -(1 << 20)
HI = (1 << 20) - 1
DISTS = ("cube", "ball", "sphere", "gauss")
SEED_BASE = 12051171 * 10


def seed_for(config_id: int) -> int:
    return SEED_BASE + int(config_id)


def _draw(dist: str, m: int, rng: np.random.Generator) -> np.ndarray:
    if dist == "cube":
        return rng.integers(LO, HI + 1, size=(m, 3), dtype=np.int64)
    if dist == "ball":
        out = np.empty((0, 3), np.int64)
        while out.shape[0] < m:
            c = rng.integers(LO, HI + 1, size=(max(2 * (m - out.shape[0]), 64), 3), dtype=np.int64)
            keep = (c * c).sum(axis=1) < (1 << 40)
            out = np.concatenate([out, c[keep]])
        return out[:m]
    if dist == "sphere":
        g = rng.standard_normal((m, 3))
        # elementwise (not a library reduction) so every platform rounds alike
        nrm = np.sqrt(g[:, 0] * g[:, 0] + g[:, 1] * g[:, 1] + g[:, 2] * g[:, 2])[:, None]
        nrm[nrm == 0] = 1.0
        return np.clip(np.rint(g / nrm * float(HI)), LO, HI).astype(np.int64)
    if dist == "gauss":
        g = np.rint(rng.standard_normal((m, 3)) * float(1 << 18))
        return np.clip(g, LO, HI).astype(np.int64)
    raise ValueError(f"unknown distribution {dist!r}")


def _key(p: np.ndarray) -> np.ndarray:
    q = p.astype(np.int64) - LO
    return (q[:, 0] << 42) | (q[:, 1] << 21) | q[:, 2]


def cloud(dist: str, n: int, rng: np.random.Generator) -> np.ndarray:
    """n distinct points of one distribution, as an (n, 3) int32 array."""
    pts = _draw(dist, n, rng)
    for _ in range(1000):
        _, first = np.unique(_key(pts), return_index=True)
        if first.size == n:
            break
        pts = np.concatenate([pts[np.sort(first)], _draw(dist, n - first.size, rng)])
    else:  # pragma: no cover
        raise RuntimeError("could not draw distinct points")
    return np.ascontiguousarray(pts, dtype=np.int32)


def cloud_seeded(dist: str, n: int, seed: int) -> np.ndarray:
    return cloud(dist, n, np.random.Generator(np.random.PCG64(seed)))


def batch_sizes(count: int, lo_exp: float, hi_exp: float, rng: np.random.Generator) -> np.ndarray:
    """Cloud sizes round(2^U(lo_exp, hi_exp))."""
    return np.rint(2.0 ** rng.uniform(lo_exp, hi_exp, size=count)).astype(np.int64)


def batch(count: int, seed: int, lo_exp: float = 4.0, hi_exp: float = 12.0):
    """A batch of independent clouds with log-uniform sizes and a distribution
    drawn uniformly from DISTS per cloud.

    Returns (xyz (N, 3) int32 concatenated, offsets (count + 1,) int64, dists)."""
    root = np.random.SeedSequence(seed)
    rng = np.random.Generator(np.random.PCG64(root))
    sizes = batch_sizes(count, lo_exp, hi_exp, rng)
    kinds = rng.integers(0, len(DISTS), size=count)
    children = root.spawn(count)
    parts = []
    for i in range(count):
        parts.append(cloud(DISTS[kinds[i]], int(sizes[i]), np.random.Generator(np.random.PCG64(children[i]))))
    offsets = np.zeros(count + 1, np.int64)
    offsets[1:] = np.cumsum(sizes)
    xyz = np.concatenate(parts) if parts else np.zeros((0, 3), np.int32)
    return np.ascontiguousarray(xyz, dtype=np.int32), offsets, [DISTS[k] for k in kinds]


PLANAR = ("square", "disk", "gauss", "grid")
PLIM = (1 << 15) - 1


def _draw2(kind: str, m: int, rng: np.random.Generator) -> np.ndarray:
    if kind == "square":
        return rng.integers(-PLIM, PLIM + 1, size=(m, 2), dtype=np.int64)
    if kind == "disk":
        out = np.empty((0, 2), np.int64)
        while out.shape[0] < m:
            c = rng.integers(-PLIM, PLIM + 1, size=(max(2 * (m - out.shape[0]), 64), 2), dtype=np.int64)
            out = np.concatenate([out, c[(c * c).sum(axis=1) < PLIM * PLIM]])
        return out[:m]
    if kind == "gauss":
        return np.clip(np.rint(rng.standard_normal((m, 2)) * float(1 << 13)), -PLIM, PLIM).astype(np.int64)
    raise ValueError(f"unknown planar distribution {kind!r}")


def planar(kind: str, n: int, rng: np.random.Generator) -> np.ndarray:
    """n distinct planar points of one kind, as an (n, 2) int32 array."""
    if kind == "grid":
        side = int(np.ceil(np.sqrt(n)))
        step = max(1, min(int(rng.integers(1, 64)), (2 * PLIM) // max(side, 1)))
        org = rng.integers(-PLIM, PLIM - step * side + 1, size=2)
        g = np.stack(np.meshgrid(np.arange(side), np.arange(side), indexing="ij"), -1).reshape(-1, 2)[:n]
        pts = org + step * g
        return np.ascontiguousarray(pts[rng.permutation(n)], dtype=np.int32)
    pts = _draw2(kind, n, rng)
    for _ in range(1000):
        _, first = np.unique(pts[:, 0] * (1 << 17) + pts[:, 1], return_index=True)
        if first.size == n:
            break
        pts = np.concatenate([pts[np.sort(first)], _draw2(kind, n - first.size, rng)])
    else:  # pragma: no cover
        raise RuntimeError("could not draw distinct points")
    return np.ascontiguousarray(pts, dtype=np.int32)


def planar_seeded(kind: str, n: int, seed: int) -> np.ndarray:
    return planar(kind, n, np.random.Generator(np.random.PCG64(seed)))
