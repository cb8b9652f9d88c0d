"""Pins of the oracle's 2D Delaunay triangulation through the lifting map
(the lower hull of (x, y, x^2 + y^2) by the method's lower pass, Sec. 2):
scipy's Delaunay (qhull) on sets in general position, the empty-circle
definition by brute force on tiny sets (exact incircle determinants), and on
degenerate sets (grids, cocircular and collinear points) the properties any
Delaunay triangulation has: every triangle counter-clockwise with positive
area, no point strictly inside a circumcircle, the triangles tiling the convex
hull (areas and edges), 2n - h - 2 triangles."""
import itertools

import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def _area2(P, a, b, c):
    return int((P[b][0] - P[a][0]) * (P[c][1] - P[a][1]) - (P[c][0] - P[a][0]) * (P[b][1] - P[a][1]))


def _incircle(P, a, b, c, d):
    """> 0 when d is strictly inside the circumcircle of the counter-clockwise (a, b, c)."""
    rows = []
    for p in (a, b, c):
        dx, dy = int(P[p][0]) - int(P[d][0]), int(P[p][1]) - int(P[d][1])
        rows.append((dx, dy, dx * dx + dy * dy))
    (a1, a2, a3), (b1, b2, b3), (c1, c2, c3) = rows
    return a1 * (b2 * c3 - b3 * c2) - a2 * (b1 * c3 - b3 * c1) + a3 * (b1 * c2 - b2 * c1)


def _canon(tris, P):
    out = []
    for a, b, c in tris:
        if _area2(P, a, b, c) < 0:
            b, c = c, b
        f = [int(a), int(b), int(c)]
        while not (f[0] < f[1] and f[0] < f[2]):
            f = f[1:] + f[:1]
        out.append(tuple(f))
    return sorted(out)


def _hull_boundary(P):
    """Points on the convex hull boundary (collinear ones included), monotone chain."""
    pts = sorted(set((int(x), int(y)) for x, y in P))

    def cross(o, a, b):
        return (a[0] - o[0]) * (b[1] - o[1]) - (a[1] - o[1]) * (b[0] - o[0])

    def chain(seq):
        h = []
        for p in seq:
            while len(h) >= 2 and cross(h[-2], h[-1], p) < 0:  # keep collinear points
                h.pop()
            h.append(p)
        return h

    lower, upper = chain(pts), chain(pts[::-1])
    ring = lower[:-1] + upper[:-1]
    area2 = sum(ring[i][0] * ring[(i + 1) % len(ring)][1] - ring[(i + 1) % len(ring)][0] * ring[i][1]
                for i in range(len(ring)))
    return set(ring), abs(area2)


def _check_triangulation(P, tris):
    n = len(P)
    assert all(_area2(P, *t) > 0 for t in tris), "every triangle counter-clockwise with positive area"
    for t in tris:
        for d in range(n):
            if d not in t:
                assert _incircle(P, *t, d) <= 0, (t, d)
    boundary, hull_area2 = _hull_boundary(P)
    assert sum(_area2(P, *t) for t in tris) == hull_area2
    edges = {}
    for t in tris:
        for k in range(3):
            e = (t[k], t[(k + 1) % 3])
            assert e not in edges, "an edge held twice in one direction"
            edges[e] = True
    if len({(int(x), int(y)) for x, y in P}) >= 3 and hull_area2 > 0:
        assert len(tris) == 2 * n - len(boundary) - 2


def test_matches_scipy_in_general_position():
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(11)
    for n in (4, 10, 100, 1000, 5000):
        pts = rng.integers(-30000, 30001, (n, 2)).astype(np.int32)
        pts = np.unique(pts, axis=0)
        rng.shuffle(pts)
        got = oracle.delaunay(pts)
        want = _canon(spatial.Delaunay(pts.astype(np.float64)).simplices, pts.astype(np.int64))
        assert sorted(map(tuple, got.tolist())) == want, n


def test_empty_circle_brute_force_in_general_position():
    rng = np.random.default_rng(12)
    done = 0
    while done < 60:
        n = int(rng.integers(3, 11))
        P = rng.integers(-50, 51, (n, 2))
        if len({tuple(p) for p in P.tolist()}) < n:
            continue
        # general position: no three collinear, no four cocircular
        if any(_area2(P, *t) == 0 for t in itertools.combinations(range(n), 3)):
            continue
        cocirc = False
        for t in itertools.combinations(range(n), 3):
            a, b, c = t if _area2(P, *t) > 0 else (t[0], t[2], t[1])
            if any(_incircle(P, a, b, c, d) == 0 for d in range(n) if d not in t):
                cocirc = True
                break
        if cocirc:
            continue
        want = []
        for t in itertools.combinations(range(n), 3):
            a, b, c = t if _area2(P, *t) > 0 else (t[0], t[2], t[1])
            if all(_incircle(P, a, b, c, d) < 0 for d in range(n) if d not in t):
                want.append((a, b, c))
        got = oracle.delaunay(P.astype(np.int32))
        assert sorted(map(tuple, got.tolist())) == _canon(want, P)
        done += 1


@pytest.mark.parametrize("case", ["grid", "square", "circle", "collinear_runs", "tiny_box"])
def test_degenerate_sets_give_a_delaunay_triangulation(case):
    rng = np.random.default_rng(13)
    if case == "grid":
        sets = [np.array([(x, y) for x in range(-4, 5) for y in range(-3, 4)])]
    elif case == "square":
        sets = [np.array([(0, 0), (1, 0), (1, 1), (0, 1)]), np.array([(-7, -7), (7, -7), (7, 7), (-7, 7), (0, 0)])]
    elif case == "circle":  # the integer points of x^2 + y^2 = 25 (all cocircular) and the centre
        ring = [(x, y) for x in range(-5, 6) for y in range(-5, 6) if x * x + y * y == 25]
        sets = [np.array(ring), np.array(ring + [(0, 0)])]
    elif case == "collinear_runs":
        sets = [np.array([(x, 0) for x in range(6)] + [(x, 5) for x in range(6)] + [(2, 2), (3, 3)])]
    else:  # many points in a tiny box: every kind of tie
        sets = []
        for _ in range(40):
            P = np.unique(rng.integers(-2, 3, (int(rng.integers(4, 20)), 2)), axis=0)
            rng.shuffle(P)
            if len(P) >= 3:
                sets.append(P)
    for P in sets:
        tris = [tuple(t) for t in oracle.delaunay(P.astype(np.int32)).tolist()]
        _check_triangulation(P, tris)


def test_square_takes_one_diagonal_and_the_result_is_deterministic():
    P = np.array([(0, 0), (2, 0), (2, 2), (0, 2)], np.int32)
    t = oracle.delaunay(P)
    assert len(t) == 2 and np.array_equal(t, oracle.delaunay(P))
    diag = set(map(tuple, t.tolist()))
    assert diag in ({(0, 1, 2), (0, 2, 3)}, {(0, 1, 3), (1, 2, 3)})


def test_range_and_duplicates_are_rejected():
    ok = np.array([[32767, -32767], [0, 0], [5, 9]], np.int32)
    assert len(oracle.delaunay(ok)) == 1
    with pytest.raises(oracle.OracleError) as e:
        oracle.delaunay(np.array([[32768, 0], [0, 0], [5, 9]], np.int32))
    assert e.value.code == 2
    with pytest.raises(oracle.OracleError) as e:
        oracle.delaunay(np.array([[1, 2], [0, 0], [1, 2]], np.int32))
    assert e.value.code == 3
    assert len(oracle.delaunay(np.array([[1, 2], [0, 0]], np.int32))) == 0
    assert len(oracle.delaunay(np.array([[0, 0], [1, 1], [2, 2]], np.int32))) == 0  # collinear: no triangle
