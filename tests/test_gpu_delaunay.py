"""2D Delaunay triangulation on the GPU through the lifting map
(hull3d_delaunay_async: the hull pipeline's lower pass on (x, y, x^2 + y^2)),
element by element against the oracle's triangulation on seeded planar sets
of every kind, ragged sizes, degenerate sets (lattices with every four
neighbours cocircular, collinear runs, tiny boxes), and the input errors."""
import numpy as np
import pytest

import oracle
from paper_1205_1171_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1205_1171_gb300 import build, hull3d

    build.build()
    oracle.build()
    return hull3d


@pytest.fixture(scope="module")
def plan(H):
    p = H.Hull3D(1 << 20)
    yield p
    p.close()


def _same(plan, pts):
    got = plan.delaunay(torch.from_numpy(np.ascontiguousarray(pts, dtype=np.int32)).cuda()).cpu().numpy()
    want = oracle.delaunay(pts)
    assert got.shape == want.shape and np.array_equal(got, want), (len(pts), got.shape, want.shape)
    return got


@pytest.mark.parametrize("kind", inputs.PLANAR)
def test_planar_sets_match_the_oracle(plan, kind):
    for i, n in enumerate((3, 4, 5, 17, 100, 1000, 4097, 10000, 65536)):
        _same(plan, inputs.planar_seeded(kind, n, 300 + i))


def test_a_million_points(plan):
    t = _same(plan, inputs.planar_seeded("disk", 1 << 20, 333))
    assert len(t) > 2 * (1 << 20) - 3000  # 2n - h - 2 with a small hull


def test_degenerate_sets(plan):
    rng = np.random.default_rng(7)
    sets = [np.array([(x, y) for x in range(-9, 10) for y in range(-9, 10)]),
            np.array([(x, 0) for x in range(40)] + [(x, 7) for x in range(40)] + [(3, 3)]),
            np.array([(x, y) for x in range(-5, 6) for y in range(-5, 6) if x * x + y * y == 25] + [(0, 0)])]
    for _ in range(300):
        P = np.unique(rng.integers(-2, 3, (int(rng.integers(3, 25)), 2)), axis=0)
        rng.shuffle(P)
        sets.append(P)
    for P in sets:
        _same(plan, P.astype(np.int32))


def test_tall_lattice_refits_the_windows(H):
    """A lattice of eight tall columns: lifted to the paraboloid, each
    column's points lie on one parabola and most of an outer column stays on
    its child's hull, so the time windows' start hulls overflow their buffer
    in a plan sized to the input; the windows are cut again, longer, and the
    triangles still match the oracle's."""
    n = 8 * 2048
    xs, ys = np.meshgrid(np.arange(-14000, 14001, 4000), np.arange(-1024, 1024), indexing="ij")
    pts = np.stack([xs.ravel(), ys.ravel()], 1).astype(np.int32)
    pts = pts[np.random.default_rng(5).permutation(n)]
    p = H.Hull3D(n)
    try:
        _same(p, pts)
        ws = p.window_stats()
        col = {k: i for i, k in enumerate(H.WINDOW_STATS)}
        refit = ws[:, col["refit"]]
        assert refit.max() >= 2, ws[9:15].tolist()
        assert (ws[refit > 0, col["pair_overflow"]] == 0).all(), ws[9:15].tolist()
    finally:
        p.close()


def test_input_errors(H, plan):
    far = inputs.planar_seeded("square", 1000, 1).copy()
    far[5, 0] = 1 << 15
    with pytest.raises(H.Hull3DError) as e:
        plan.delaunay(torch.from_numpy(far).cuda())
    assert e.value.code == H.ERR_COORD_RANGE
    dup = inputs.planar_seeded("square", 1000, 2).copy()
    dup[7] = dup[3]
    with pytest.raises(H.Hull3DError) as e:
        plan.delaunay(torch.from_numpy(dup).cuda())
    assert e.value.code == H.ERR_DUPLICATE
    two = torch.tensor([[0, 0], [5, 5]], dtype=torch.int32, device="cuda")
    assert plan.delaunay(two).shape[0] == 0
