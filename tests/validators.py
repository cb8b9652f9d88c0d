"""Structural checks of a canonical face list, independent of how it was made.

All arithmetic is exact integer arithmetic (int64 with a split product)."""
from __future__ import annotations

import numpy as np


def euler_ok(faces: np.ndarray) -> bool:
    """F = 2V - 4 for a triangulated sphere (V = distinct vertices used)."""
    if len(faces) == 0:
        return True
    v = np.unique(faces).size
    return len(faces) == 2 * v - 4


def manifold_ok(faces: np.ndarray) -> bool:
    """Every directed edge appears exactly once and so does its reverse."""
    if len(faces) == 0:
        return True
    f = faces.astype(np.int64)
    e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]])
    key = (e[:, 0] << 32) | e[:, 1]
    rkey = (e[:, 1] << 32) | e[:, 0]
    u, cnt = np.unique(key, return_counts=True)
    if np.any(cnt != 1):
        return False
    return bool(np.all(np.isin(rkey, u)))


def canonical(faces) -> np.ndarray:
    """Rotate each oriented triangle min-first and sort the list."""
    f = np.asarray(faces, dtype=np.int64).reshape(-1, 3)
    out = f.copy()
    for _ in range(2):
        rot = ~((out[:, 0] < out[:, 1]) & (out[:, 0] < out[:, 2]))
        out[rot] = out[rot][:, [1, 2, 0]]
    order = np.lexsort((out[:, 2], out[:, 1], out[:, 0]))
    return out[order].astype(np.int32)


def _dot_sign(N: np.ndarray, D: np.ndarray) -> np.ndarray:
    """Exact sign of the row-wise dot product N . D with |N| < 2^44, |D| < 2^22."""
    nhi = N >> 22
    nlo = N & ((1 << 22) - 1)
    A = (nhi * D).sum(axis=-1)
    B = (nlo * D).sum(axis=-1)
    A2 = A + (B >> 22)
    B2 = B & ((1 << 22) - 1)
    return np.where(A2 > 0, 1, np.where(A2 < 0, -1, np.where(B2 > 0, 1, 0)))


def face_normals(pts: np.ndarray, faces: np.ndarray) -> np.ndarray:
    p = pts.astype(np.int64)
    a, b, c = p[faces[:, 0]], p[faces[:, 1]], p[faces[:, 2]]
    return np.cross(b - a, c - a)


def side_ok(pts: np.ndarray, faces: np.ndarray, chunk: int = 256) -> bool:
    """Every point is on or behind every face's (unperturbed) plane."""
    p = pts.astype(np.int64)
    N = face_normals(pts, faces)
    A = p[faces[:, 0]]
    for s in range(0, len(faces), chunk):
        n = N[s:s + chunk][:, None, :]
        d = p[None, :, :] - A[s:s + chunk][:, None, :]
        if np.any(_dot_sign(np.broadcast_to(n, d.shape), d) > 0):
            return False
    return True


def side_ok_sampled(pts: np.ndarray, faces: np.ndarray, nface: int, npts: int, seed: int = 0) -> bool:
    rng = np.random.default_rng(seed)
    fi = rng.choice(len(faces), size=min(nface, len(faces)), replace=False)
    pi = rng.choice(len(pts), size=min(npts, len(pts)), replace=False)
    verts = np.unique(faces)
    sub = np.unique(np.concatenate([pi, verts[: min(len(verts), npts)]]))
    p = pts.astype(np.int64)
    N = face_normals(pts, faces[fi])
    A = p[faces[fi, 0]]
    for s in range(0, len(fi), 64):
        n = N[s:s + 64][:, None, :]
        d = p[sub][None, :, :] - A[s:s + 64][:, None, :]
        if np.any(_dot_sign(np.broadcast_to(n, d.shape), d) > 0):
            return False
    return True


def extreme_ok(pts: np.ndarray, faces: np.ndarray, ndir: int = 64, seed: int = 0) -> bool:
    """The maximiser of a random integer direction is a hull vertex."""
    rng = np.random.default_rng(seed)
    verts = set(np.unique(faces).tolist())
    p = pts.astype(np.int64)
    for _ in range(ndir):
        d = rng.integers(-1000, 1001, size=3)
        s = p @ d
        best = np.flatnonzero(s == s.max())
        if not any(int(b) in verts for b in best):
            return False
    return True


def check_all(pts: np.ndarray, faces: np.ndarray, side: bool = True) -> None:
    n = len(pts)
    if n < 3:
        assert len(faces) == 0
        return
    assert euler_ok(faces), "Euler F = 2V - 4 fails"
    assert manifold_ok(faces), "not a closed 2-manifold"
    if side:
        assert side_ok(pts, faces), "a point lies outside a face"
