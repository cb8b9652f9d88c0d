"""Pins the oracle's hull to results fixed by the mathematics, not by itself.

* perturbed brute force (a triple is a face iff all other points lie strictly
  on one side of its perturbed plane) on thousands of tiny degenerate inputs;
* qhull (scipy) on inputs in general position, where the hull is unique;
* closed forms: the cyclic polytope's faces by Gale's evenness condition, the
  tetrahedron, octahedron and cube, and the paraboloid whose lower hull is the
  Delaunay triangulation;
* kinetic invariants of the movies (Sec. 2): strictly increasing event times,
  one contiguous hull interval per point, the t = -inf and t = +inf states;
* Euler, 2-manifold and all-points side tests at moderate sizes.
"""
from fractions import Fraction
from itertools import combinations

import numpy as np
import pytest

import oracle
from paper_1205_1171_gb300 import inputs
from tests import validators as V


def _tiny_sets(count, seed):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        kind = len(out) % 6
        n = int(rng.integers(3, 13))
        if kind == 0:  # tiny box: every degeneracy at once
            p = rng.integers(-2, 3, size=(n, 3))
        elif kind == 1:  # grid
            g = np.array(np.meshgrid(*[np.arange(3)] * 3)).reshape(3, -1).T
            p = g[rng.choice(len(g), size=min(n, len(g)), replace=False)] * rng.integers(1, 4)
        elif kind == 2:  # vertical line plus a few points
            k = int(rng.integers(2, max(3, n)))
            line = np.stack([np.zeros(k), np.zeros(k), rng.choice(np.arange(-9, 10), size=k, replace=False)], 1)
            p = np.concatenate([line, rng.integers(-3, 4, size=(n - k, 3))])
        elif kind == 3:  # coplanar slab z = const plus a few
            k = int(rng.integers(3, max(4, n)))
            slab = np.concatenate([rng.integers(-3, 4, size=(k, 2)), np.zeros((k, 1))], 1)
            p = np.concatenate([slab, rng.integers(-3, 4, size=(n - k, 3))])
        elif kind == 4:  # oblique collinear run plus a few
            d = rng.integers(-2, 3, size=3)
            if not d.any():
                continue
            k = int(rng.integers(2, max(3, n)))
            run = np.outer(np.arange(k), d)
            p = np.concatenate([run, rng.integers(-3, 4, size=(n - k, 3))])
        else:  # cube-surface points (coplanar facets, collinear edges)
            p = rng.integers(-2, 3, size=(n, 3))
            ax = rng.integers(0, 3, size=n)
            p[np.arange(n), ax] = rng.choice([-2, 2], size=n)
        p = np.unique(p.astype(np.int64), axis=0)
        if len(p) < 3:
            continue
        out.append(rng.permutation(p).astype(np.int32))
    return out


def test_trivial_sizes():
    assert len(oracle.hull(np.array([[1, 2, 3]]))) == 0
    assert len(oracle.hull(np.array([[1, 2, 3], [4, 5, 6]]))) == 0
    f = oracle.hull(np.array([[0, 0, 0], [5, 1, 2], [1, 7, 3]]))
    assert f.tolist() == [[0, 1, 2], [0, 2, 1]]


def test_errors():
    with pytest.raises(oracle.OracleError) as e:
        oracle.hull(np.array([[0, 0, 1 << 20], [1, 2, 3], [4, 5, 6]]))
    assert e.value.code == 2
    with pytest.raises(oracle.OracleError) as e:
        oracle.hull(np.array([[-(1 << 20) - 1, 0, 0], [1, 2, 3], [4, 5, 6]]))
    assert e.value.code == 2
    with pytest.raises(oracle.OracleError) as e:
        oracle.hull(np.array([[1, 2, 3], [4, 5, 6], [1, 2, 3], [0, 0, 0]]))
    assert e.value.code == 3


def _sympy_brute(pts):
    """Independent brute force on the definition (sympy orient3d), tiny n only."""
    from tests.test_oracle_predicates import ref_orient3d

    n = len(pts)
    faces = []
    ids = np.arange(n, dtype=np.int32)
    for i, j, k in combinations(range(n), 3):
        s = {ref_orient3d(pts[[i, j, k, l]], ids[[i, j, k, l]]) for l in range(n) if l not in (i, j, k)}
        if len(s) == 1:
            faces.append((i, j, k) if s.pop() < 0 else (i, k, j))
    return V.canonical(faces)


def test_brute_force_pinned_to_sympy():
    pytest.importorskip("sympy")
    for pts in _tiny_sets(12, 99)[:12]:
        if len(pts) > 7 or len(pts) < 4:
            continue
        assert np.array_equal(oracle.brute_faces(pts), _sympy_brute(pts))


@pytest.mark.parametrize("seed", range(4))
def test_matches_perturbed_brute_force(seed):
    for pts in _tiny_sets(500, seed):
        want = oracle.brute_faces(pts)
        got = oracle.hull(pts)
        assert np.array_equal(got, want), pts.tolist()
        assert np.array_equal(oracle.hull(pts, split="aligned"), want)
        V.check_all(pts, got)


def _qhull(pts):
    from scipy.spatial import ConvexHull

    h = ConvexHull(pts.astype(np.float64))
    f = h.simplices.astype(np.int64)
    nrm = V.face_normals(pts, f).astype(np.float64)
    flip = (nrm * h.equations[:, :3]).sum(1) < 0
    f[flip] = f[flip][:, [0, 2, 1]]
    return V.canonical(f)


@pytest.mark.parametrize("dist,n", [("cube", 64), ("cube", 3000), ("ball", 3000), ("sphere", 1500), ("ball", 200)])
def test_matches_qhull_general_position(dist, n):
    pts = inputs.cloud_seeded(dist, n, 1000 + n)
    got = oracle.hull(pts)
    want = _qhull(pts)
    assert np.array_equal(got, want)


def _gale_facets(n):
    """Facets of the cyclic 3-polytope on n points (Gale's evenness condition)."""
    out = []
    for S in combinations(range(n), 3):
        ok = True
        for a, b in combinations([i for i in range(n) if i not in S], 2):
            if sum(1 for s in S if a < s < b) % 2:
                ok = False
                break
        if ok:
            out.append(S)
    return out


@pytest.mark.parametrize("perm", [(0, 1, 2), (1, 0, 2), (2, 1, 0), (0, 2, 1)])
def test_cyclic_polytope_gale(perm):
    rng = np.random.default_rng(sum(perm) + 3 * perm[0])
    t = np.sort(rng.choice(np.arange(-101, 102), size=60, replace=False))
    curve = np.stack([t, t**2, t**3], 1)[:, perm]
    order = rng.permutation(len(t))
    pts = curve[order].astype(np.int32)
    pos = np.argsort(order)  # pos[i] = input index of the curve point i
    got = oracle.hull(pts)
    assert len(got) == 2 * len(t) - 4
    want = {tuple(sorted(pos[list(S)])) for S in _gale_facets(len(t))}
    assert {tuple(sorted(f)) for f in got.tolist()} == want
    V.check_all(pts, got)


def test_tetrahedron_exact():
    pts = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])
    # hand-derived outward faces: z=0 -> (0,2,1), y=0 -> (0,1,3), x=0 -> (0,3,2), slanted -> (1,2,3)
    assert oracle.hull(pts).tolist() == [[0, 1, 3], [0, 2, 1], [0, 3, 2], [1, 2, 3]]


def test_octahedron_exact():
    s = 1000
    pts = np.array([[s, 0, 0], [-s, 0, 0], [0, s, 0], [0, -s, 0], [0, 0, s], [0, 0, -s]])
    want = []
    for sx, ix in ((1, 0), (-1, 1)):
        for sy, iy in ((1, 2), (-1, 3)):
            for sz, iz in ((1, 4), (-1, 5)):
                f = (ix, iy, iz)
                nrm = np.cross(pts[iy] - pts[ix], pts[iz] - pts[ix])
                if np.dot(nrm, (sx, sy, sz)) < 0:
                    f = (ix, iz, iy)
                want.append(f)
    assert np.array_equal(oracle.hull(pts), V.canonical(want))


def test_cube_corners():
    s = 1000
    pts = np.array([[x, y, z] for x in (-s, s) for y in (-s, s) for z in (-s, s)])
    f = oracle.hull(pts)
    assert len(f) == 12 and np.unique(f).size == 8
    V.check_all(pts, f)
    for tri in f:
        p = pts[tri]
        assert any(np.all(p[:, k] == p[0, k]) for k in range(3))  # lies in a cube facet


def test_paraboloid_lower_hull_is_delaunay():
    from scipy.spatial import Delaunay

    rng = np.random.default_rng(21)
    xy = np.unique(rng.integers(-723, 724, size=(400, 2)), axis=0)
    xy = rng.permutation(xy)
    pts = np.concatenate([xy, (xy**2).sum(1, keepdims=True)], 1).astype(np.int32)
    f = oracle.hull(pts)
    V.check_all(pts, f)
    nz = V.face_normals(pts, f)[:, 2]
    assert np.all(nz != 0)
    lower = {tuple(sorted(t)) for t in f[nz < 0].tolist()}
    tri = Delaunay(xy.astype(np.float64))
    # degeneracy check: no Delaunay edge has its two opposite vertices cocircular
    P = [tuple(int(v) for v in r) for r in pts]

    def incircle(a, b, c, d):
        m = [[P[k][0] - P[d][0], P[k][1] - P[d][1], P[k][2] - P[d][2]] for k in (a, b, c)]
        return (m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0])
                + m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]))

    for s, nb in zip(tri.simplices, tri.neighbors):
        for k in range(3):
            if nb[k] >= 0:
                d = [v for v in tri.simplices[nb[k]] if v not in s][0]
                assert incircle(int(s[0]), int(s[1]), int(s[2]), int(d)) != 0
    assert lower == {tuple(sorted(int(v) for v in t)) for t in tri.simplices}


def _exact_time(P, a, w, b):
    Y = (P[w][0] - P[a][0]) * (P[b][1] - P[a][1]) - (P[b][0] - P[a][0]) * (P[w][1] - P[a][1])
    Z = (P[w][0] - P[a][0]) * (P[b][2] - P[a][2]) - (P[b][0] - P[a][0]) * (P[w][2] - P[a][2])
    assert Y != 0
    return Fraction(Z, Y)


def _monotone_chain(P, idx, upper):
    """Plain lower (or upper) hull of points already in x order (rank lists)."""
    out = []
    for i in idx:
        while len(out) >= 2:
            a, b = out[-2], out[-1]
            cr = (P[b][0] - P[a][0]) * (P[i][1] - P[a][1]) - (P[i][0] - P[a][0]) * (P[b][1] - P[a][1])
            if (cr <= 0) if not upper else (cr >= 0):
                out.pop()
            else:
                break
        out.append(i)
    return out


@pytest.mark.parametrize("upper", [False, True])
def test_kinetic_invariants(upper):
    pts = inputs.cloud_seeded("cube", 600, 31)
    order = oracle.sort_order(pts)
    P = [tuple(int(v) for v in pts[i]) for i in order]  # by rank
    rng = np.random.default_rng(5)
    nodes = [(0, 600), (0, 300), (300, 600), (17, 40), (128, 256)]
    nodes += [tuple(sorted(rng.choice(600, 2, replace=False).tolist())) for _ in range(10)]
    for lo, hi in nodes:
        if hi - lo < 4:
            continue
        w, a, b, ins, neg = oracle.node_events(pts, lo, hi, upper)
        m = hi - lo
        assert len(w) <= 2 * m - 5
        # strictly monotone event times (the z-mirrored pass runs time backwards)
        ts = [_exact_time(P, a[k], w[k], b[k]) for k in range(len(w))]
        for k in range(1, len(ts)):
            assert (ts[k] < ts[k - 1]) if upper else (ts[k] > ts[k - 1])
        # t = -inf hull is the xy lower hull
        assert neg.tolist() == _monotone_chain(P, range(lo, hi), upper=False)
        # replay: one contiguous interval per point, and the +inf state
        alive = list(neg.tolist())
        seen = {}
        for k in range(len(w)):
            p = int(w[k])
            seen.setdefault(p, []).append(bool(ins[k]))
            if ins[k]:
                j = alive.index(int(a[k]))
                assert alive[j + 1] == b[k]
                alive.insert(j + 1, p)
            else:
                j = alive.index(p)
                assert alive[j - 1] == a[k] and alive[j + 1] == b[k]
                alive.pop(j)
        for p, kinds in seen.items():
            assert kinds in ([True], [False], [True, False]), (p, kinds)
            if kinds[0]:
                assert p not in neg
        assert alive == _monotone_chain(P, range(lo, hi), upper=True)


@pytest.mark.parametrize("dist", inputs.DISTS)
def test_structural_invariants_moderate(dist):
    for n in (5, 33, 257, 2000):
        pts = inputs.cloud_seeded(dist, n, 77 + n)
        f = oracle.hull(pts)
        V.check_all(pts, f)
        assert V.extreme_ok(pts, f)
        assert np.array_equal(f, oracle.hull(pts, split="aligned"))


def test_sort_order_is_lexicographic_xzy():
    pts = inputs.cloud_seeded("gauss", 5000, 3)
    want = np.lexsort((pts[:, 1], pts[:, 2], pts[:, 0]))
    assert np.array_equal(oracle.sort_order(pts), want)
