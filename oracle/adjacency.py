"""CPU oracle of the hull's adjacency (test infrastructure, like the rest of
``oracle/``).

The paper names an arrangement structure such as a doubly connected edge list
as the prerequisite for further geometry on the GPU (Sec. 5).  For a convex
hull given as its canonical face list (outward counter-clockwise triples of
input indices) that structure is fixed by two relations, written out here by
their plain definitions with dictionaries and loops:

* face neighbours: edge k of face f runs from f[k] to f[(k + 1) % 3]; on a
  closed, consistently oriented surface exactly one other face holds the same
  edge in the opposite direction, and ``nb[f, k]`` is that face;
* vertex stars: the faces around a vertex v in counter-clockwise order seen
  from outside.  Around v, face (v, a, b) is followed by the face that holds
  the edge v -> b, i.e. the neighbour of (v, a, b) across its edge b -> v.
  Each star starts at the smallest face index around v; vertices on no face
  (interior points) have empty stars.  The stars are returned in CSR form:
  ``star[off[v]:off[v + 1]]``.
"""
from __future__ import annotations

import numpy as np


def face_neighbors(faces) -> np.ndarray:
    """(F, 3) int32: ``nb[f, k]`` is the face holding the directed edge
    (f[(k + 1) % 3], f[k]).  Raises ValueError where an edge is held twice in
    one direction or its opposite is missing (not a closed oriented surface)."""
    faces = np.asarray(faces, dtype=np.int64).reshape(-1, 3)
    owner = {}
    for f, tri in enumerate(faces.tolist()):
        for k in range(3):
            e = (tri[k], tri[(k + 1) % 3])
            if e in owner:
                raise ValueError(f"directed edge {e} held by faces {owner[e]} and {f}")
            owner[e] = f
    nb = np.empty(faces.shape, dtype=np.int32)
    for f, tri in enumerate(faces.tolist()):
        for k in range(3):
            opp = (tri[(k + 1) % 3], tri[k])
            if opp not in owner:
                raise ValueError(f"edge {opp[::-1]} of face {f} has no opposite face")
            nb[f, k] = owner[opp]
    return nb


def vertex_stars(faces, n: int) -> tuple[np.ndarray, np.ndarray]:
    """CSR vertex stars of the hull of n points: (off int64[n + 1], star
    int32[3F]).  Raises ValueError if the faces around a vertex do not form
    one cycle."""
    faces = np.asarray(faces, dtype=np.int64).reshape(-1, 3)
    nb = face_neighbors(faces)
    around = [[] for _ in range(n)]
    for f, tri in enumerate(faces.tolist()):
        for v in tri:
            around[v].append(f)
    off = np.zeros(n + 1, dtype=np.int64)
    star = np.empty(3 * len(faces), dtype=np.int32)
    pos = 0
    for v in range(n):
        if around[v]:
            first = min(around[v])
            f = first
            while True:
                star[pos] = f
                pos += 1
                tri = faces[f].tolist()
                k = tri.index(v)
                # (v, a, b) = tri rotated to v; the edge b -> v is edge (k + 2) % 3
                f = int(nb[f, (k + 2) % 3])
                if f == first:
                    break
                if pos - off[v] > len(around[v]):
                    raise ValueError(f"faces around vertex {v} do not close")
            if pos - off[v] != len(around[v]):
                raise ValueError(f"faces around vertex {v} form more than one cycle")
        off[v + 1] = pos
    return off, star
