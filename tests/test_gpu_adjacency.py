"""Adjacency of the hull on the GPU (hull3d_adjacency_async): the face across
each directed edge and the counter-clockwise vertex stars, the arrangement
structure of Sec. 5, element by element against the oracle's plain
definitions (oracle/adjacency.py) on the hand-derived tetrahedron, on hulls of
every distribution at 2^16 and 2^20 points, and on the error cases."""
import numpy as np
import pytest

import oracle
from oracle import adjacency
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


def _check(faces_np, nb, off, star, n):
    want_nb = adjacency.face_neighbors(faces_np)
    want_off, want_star = adjacency.vertex_stars(faces_np, n)
    assert np.array_equal(nb.cpu().numpy(), want_nb)
    assert np.array_equal(off.cpu().numpy(), want_off)
    assert np.array_equal(star.cpu().numpy(), want_star)


def test_tetrahedron_by_hand(H):
    pts = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], np.int32)
    plan = H.Hull3D(4)
    try:
        faces = plan.compute(torch.from_numpy(pts).cuda())
        nb, off, star = plan.adjacency(faces, 4)
        assert nb.cpu().tolist() == [[1, 3, 2], [2, 3, 0], [0, 3, 1], [1, 2, 0]]
        assert off.cpu().tolist() == [0, 3, 6, 9, 12]
        assert star.cpu().tolist() == [0, 2, 1, 0, 1, 3, 1, 2, 3, 0, 3, 2]
    finally:
        plan.close()


@pytest.mark.parametrize("n", [1 << 16, 1 << 20])
@pytest.mark.parametrize("dist", inputs.DISTS)
def test_adjacency_matches_the_oracle(H, dist, n):
    pts = inputs.cloud_seeded(dist, n, inputs.seed_for(7) + n)
    plan = H.Hull3D(n)
    try:
        faces = plan.compute(torch.from_numpy(pts).cuda())
        f = faces.cpu().numpy()
        if n <= 1 << 16:  # the face list itself (the larger sizes are checked in the parity tests)
            assert np.array_equal(f, oracle.hull(pts))
        nb, off, star = plan.adjacency(faces, n)
        _check(f, nb, off, star, n)
        # twice in a row on the same plan: the scratch keeps no state
        nb2, off2, star2 = plan.adjacency(faces, n)
        assert torch.equal(nb, nb2) and torch.equal(off, off2) and torch.equal(star, star2)
    finally:
        plan.close()


def test_open_or_doubled_surfaces_are_rejected(H):
    pts = inputs.cloud_seeded("cube", 300, 7)
    plan = H.Hull3D(300)
    try:
        faces = plan.compute(torch.from_numpy(pts).cuda())
        with pytest.raises(H.Hull3DError) as e:
            plan.adjacency(faces[1:].contiguous(), 300)  # one face missing: its edges have no opposite
        assert e.value.code == H.ERR_NOT_CLOSED
        with pytest.raises(H.Hull3DError) as e:
            plan.adjacency(torch.cat([faces, faces[:1]]).contiguous(), 300)  # one face twice
        assert e.value.code == H.ERR_NOT_CLOSED
        # every face reversed is still a closed, consistently oriented surface
        rev = faces.flip(1).contiguous()
        nb, off, star = plan.adjacency(rev, 300)
        _check(rev.cpu().numpy(), nb, off, star, 300)
    finally:
        plan.close()


def test_no_faces_gives_empty_stars(H):
    plan = H.Hull3D(8)
    try:
        faces = torch.zeros((0, 3), dtype=torch.int32, device="cuda")
        nb, off, star = plan.adjacency(faces, 2)
        assert nb.shape == (0, 3) and off.cpu().tolist() == [0, 0, 0] and star.numel() == 0
    finally:
        plan.close()
