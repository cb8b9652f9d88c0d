"""Pins of the adjacency oracle (face neighbours and vertex stars of the
canonical hull, the arrangement structure of Sec. 5): a hand-derived
tetrahedron, the octahedron's face graph (the cube graph), invariants on hulls
of every distribution, and rejection of a surface that is not closed."""
import numpy as np
import pytest

import oracle
from oracle import adjacency
from paper_1205_1171_gb300 import inputs


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def test_tetrahedron_by_hand():
    # vertices 0:(0,0,0) 1:(1,0,0) 2:(0,1,0) 3:(0,0,1); outward normals
    # (0,1,3): -y, (0,2,1): -z, (0,3,2): -x, (1,2,3): (1,1,1)
    pts = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], np.int32)
    faces = oracle.hull(pts)
    assert faces.tolist() == [[0, 1, 3], [0, 2, 1], [0, 3, 2], [1, 2, 3]]
    nb = adjacency.face_neighbors(faces)
    # nb[f, k]: the face across edge f[k] -> f[k+1]
    assert nb.tolist() == [[1, 3, 2], [2, 3, 0], [0, 3, 1], [1, 2, 0]]
    off, star = adjacency.vertex_stars(faces, 4)
    assert off.tolist() == [0, 3, 6, 9, 12]
    # counter-clockwise seen from outside, from the smallest face: at vertex 0
    # the faces run through the x, z, y directions in turn
    assert star.tolist() == [0, 2, 1, 0, 1, 3, 1, 2, 3, 0, 3, 2]


def test_octahedron_face_graph_is_the_cube_graph():
    r = 1000
    pts = np.array([[r, 0, 0], [-r, 0, 0], [0, r, 0], [0, -r, 0], [0, 0, r], [0, 0, -r]], np.int32)
    faces = oracle.hull(pts)
    assert len(faces) == 8

    def octant(tri):  # the sign triple of the face's centroid
        c = pts[tri].sum(axis=0)
        return tuple(int(np.sign(v)) for v in c)

    octs = [octant(t) for t in faces]
    assert len(set(octs)) == 8
    nb = adjacency.face_neighbors(faces)
    for f in range(8):
        got = sorted(octs[g] for g in nb[f])
        want = sorted(tuple(-s if i == j else s for i, s in enumerate(octs[f])) for j in range(3))
        assert got == want
    off, star = adjacency.vertex_stars(faces, 6)
    assert np.diff(off).tolist() == [4] * 6


@pytest.mark.parametrize("dist,n", [("cube", 3000), ("ball", 2000), ("sphere", 1500), ("gauss", 4000)])
def test_invariants_on_hulls(dist, n):
    pts = inputs.cloud_seeded(dist, n, 90 + n)
    faces = oracle.hull(pts)
    F = len(faces)
    nb = adjacency.face_neighbors(faces)
    for f in range(F):
        for k in range(3):
            g = int(nb[f, k])
            assert g != f
            a, b = faces[f, k], faces[f, (k + 1) % 3]
            # g holds b -> a, and its neighbour across that edge is f
            j = [int(x) for x in range(3) if faces[g, x] == b and faces[g, (x + 1) % 3] == a]
            assert len(j) == 1 and nb[g, j[0]] == f
    off, star = adjacency.vertex_stars(faces, n)
    assert off[-1] == 3 * F
    deg = np.bincount(faces.ravel(), minlength=n)
    assert np.array_equal(np.diff(off), deg)
    for v in np.flatnonzero(deg):
        s = star[off[v]: off[v + 1]]
        assert s[0] == s.min()
        for i in range(len(s)):  # consecutive faces share an edge at v
            f, g = faces[s[i]], faces[s[(i + 1) % len(s)]]
            shared = set(f.tolist()) & set(g.tolist())
            assert v in shared and len(shared) == 2


def test_open_surface_is_rejected():
    pts = inputs.cloud_seeded("cube", 200, 7)
    faces = oracle.hull(pts)
    with pytest.raises(ValueError):
        adjacency.face_neighbors(faces[1:])
    with pytest.raises(ValueError):
        adjacency.face_neighbors(np.concatenate([faces, faces[:1]]))
